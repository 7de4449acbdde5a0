// Internal declarations shared by the translation units of libgbh.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "gbh.h"

namespace gbh {

constexpr int kMaxDim = 16;
constexpr int kMaxLevel = 30;

// Geometry of one grid: levels, extents n_k = 2^{l_k}+1, strides S_k.
struct Geom {
    int d;
    int l[kMaxDim];
    int64_t n[kMaxDim];
    int64_t S[kMaxDim];
    int64_t N;       // points of one grid
    int64_t batch;   // grids of this shape stored back to back (>= 1)
    int64_t total;   // batch * N
};

// Validates (d, levels) and fills g; returns GBH_OK or an error status.
int make_geom(int d, const int32_t *levels, int elem_size, Geom *g);

// Adds `k` to the process-wide count of kernels launched by the library.
void count_launches(uint64_t k);

// Optional per-launch event timing (gbh_profile_*): construct before a launch,
// call done() after it.  Does nothing while profiling is off.
class ProfScope {
  public:
    ProfScope(const char *name, cudaStream_t s, double alg_bytes);
    void done();
  private:
    const char *name_;
    cudaStream_t s_;
    double bytes_;
    void *ev0_ = nullptr;
};

// Maps the last CUDA error (if any) to a status; clears sticky-free errors.
int check_launch();

// Number of SMs of the current device (cached per device).
int num_sms();

// Grouped path: one pass per group of consecutive dimensions whose pole sets
// fit in a shared-memory tile (hierarchize and dehierarchize).  Returns
// GBH_EUNSUPPORTED for shapes it does not take.
int grouped_transform(void *data, const Geom &g, int dtype, int op, cudaStream_t s);

// Plain path: one sweep per dimension.  fixed64: fp64 pole groups compute in
// int64 fixed point (otherwise native arithmetic in the serial operation
// order, bit-identical to the serial algorithm).  pairs: with native
// arithmetic, two consecutive dimensions per pass where their poles fit a
// pair tile (same results, one memory crossing fewer per pair).
// short_native: with fixed64, dimensions of level 1 compute natively (and may
// pair); the default route asks for it, an explicit fixed-point request not.
int plain_transform(void *data, const Geom &g, int dtype, int op, cudaStream_t s, bool fixed64 = false,
                    bool pairs = true, bool short_native = false);

// Fused path: dyadic tiles (class-ordered), see fused.cu.
int fused_transform(void *data, const Geom &g, int dtype, int op, const gbh_options *opt,
                    cudaStream_t s);

// Interior class of the fused path for 3-D fp64 grids in fixed point with
// tile exponents (5,4,4), one closure per CTA (interior3.cu).  Returns 1
// (nothing launched) when the shape is not one it takes.
bool interior3_applicable(const Geom &g, const int *m);
int interior3_transform(double *u, const Geom &g, const int *m, int op, cudaStream_t s);

// Tile exponents the fused path would choose (false if unsupported).
bool fused_tiles(const Geom &g, int dtype, int op, int *m_out);

// True if the planner would rather run the fused path than the plain one
// (estimated DRAM bytes well below one sweep per dimension).
bool fused_preferred(const Geom &g, int dtype, int op);

// True if the fused path supports this (geometry, dtype, op).
bool fused_supported(const Geom &g, int dtype, int op);

// Up to K feasible tile-exponent vectors of the fused path, best estimate
// first (false if the fused path does not take the shape).
bool fused_candidates(const Geom &g, int dtype, int op, int K, std::vector<std::vector<int>> *out);

// Makes tile exponents m the fused path's choice for this shape (autotuner);
// fused_forget_pins drops every choice (the cost model decides again).
bool fused_pin_tiles(const Geom &g, int dtype, int op, const int *m);
void fused_forget_pins();

// Execution path the autotuner recorded for this shape (gbh_path), or -1.
int tuned_path(const Geom &g, int dtype, int op);

// Fills n values of dtype at u with scratch values in [-1, 1) (timing data).
int launch_fill(void *u, int64_t n, int dtype, unsigned seed, cudaStream_t s);

}  // namespace gbh
