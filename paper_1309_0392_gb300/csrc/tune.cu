// Autotuner of the single-grid transform: the execution path (one sweep per
// dimension, dyadic tiles, or dimension groups) and the tile shape of the
// dyadic path are chosen per level vector by timing the candidates on a
// scratch grid of that shape, instead of by the DRAM-byte cost model alone.
// The choice is kept in a process-wide table keyed by (d, levels, dtype, op)
// that the default path consults.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "gbh_internal.h"

namespace gbh {
namespace {

std::mutex g_tune_mu;
std::map<std::vector<int>, int> g_tuned_path;    // key -> gbh_path

std::vector<int> tune_key(const Geom &g, int dtype, int op)
{
    std::vector<int> key{g.d, dtype, op};
    for (int k = 0; k < g.d; ++k) key.push_back(g.l[k]);
    return key;
}

// Scratch values in [-1, 1) from a hash of the index (timing data only).
template <typename T>
__global__ void k_fill(T *u, int64_t n, unsigned seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ull + seed;
        h ^= h >> 31;
        h *= 0xBF58476D1CE4E5B9ull;
        h ^= h >> 29;
        u[i] = (T)((double)(h >> 11) * (1.0 / 4503599627370496.0) - 1.0);
    }
}

struct Candidate {
    int path;
    std::vector<int> m;
};

}  // namespace

int launch_fill(void *u, int64_t n, int dtype, unsigned seed, cudaStream_t s)
{
    if (n <= 0) return GBH_OK;
    const int grid = std::max(1, std::min<int>(num_sms() * 8, (int)((n + 255) / 256)));
    if (dtype == GBH_F64) k_fill<double><<<grid, 256, 0, s>>>(static_cast<double *>(u), n, seed);
    else k_fill<float><<<grid, 256, 0, s>>>(static_cast<float *>(u), n, seed);
    return check_launch();
}

int tuned_path(const Geom &g, int dtype, int op)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_path.find(tune_key(g, dtype, op));
    return it == g_tuned_path.end() ? -1 : it->second;
}

}  // namespace gbh

using namespace gbh;

extern "C" int gbh_autotune(int d, const int32_t *levels, int dtype, int op, gbh_tune_result *out)
{
    if (!out) return GBH_EINVAL;
    if (dtype != GBH_F32 && dtype != GBH_F64) return GBH_EDTYPE;
    if (op != GBH_HIERARCHIZE && op != GBH_DEHIERARCHIZE && op != GBH_ADJOINT && op != GBH_DEHIERARCHIZE_ADJOINT)
        return GBH_EINVAL;
    const int es = dtype == GBH_F64 ? 8 : 4;
    Geom g;
    if (int e = make_geom(d, levels, es, &g)) return e;
    std::memset(out, 0, sizeof(*out));

    // the cost model's choice (what the default path runs untuned)
    Candidate model{GBH_PATH_PLAIN, {}};
    if (g.N >= 4096 && fused_preferred(g, dtype, op)) {
        int m[kMaxDim] = {0};
        fused_tiles(g, dtype, op, m);
        model = Candidate{GBH_PATH_FUSED, std::vector<int>(m, m + d)};
    }
    // candidates: the per-dimension sweeps, the best-estimated tiles of the
    // fused path, and the dimension groups
    std::vector<Candidate> cands{Candidate{GBH_PATH_PLAIN, {}}};
    std::vector<std::vector<int>> tiles;
    if (fused_candidates(g, dtype, op, 6, &tiles))
        for (auto &m : tiles) cands.push_back(Candidate{GBH_PATH_FUSED, m});
    if (op == GBH_HIERARCHIZE || op == GBH_DEHIERARCHIZE) cands.push_back(Candidate{GBH_PATH_GROUPED, {}});

    void *buf = nullptr, *pristine = nullptr;
    const size_t bytes = (size_t)g.N * es;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return GBH_ENOMEM;
    if (cudaMalloc(&pristine, bytes) != cudaSuccess) {
        cudaFree(buf);
        return GBH_ENOMEM;
    }
    cudaStream_t s;
    cudaEvent_t e0, e1;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch_fill(pristine, g.N, dtype, 12345u, s);

    auto run = [&](const Candidate &c) -> int {
        gbh_options opt;
        std::memset(&opt, 0, sizeof(opt));
        opt.path = c.path;
        // fp64 sweeps in fixed point, as the default path runs them
        opt.arith = (c.path == GBH_PATH_PLAIN && dtype == GBH_F64) ? 2 : 0;
        for (size_t k = 0; k < c.m.size(); ++k) opt.tile_exp[k] = c.m[k];
        return gbh_transform(buf, d, levels, dtype, op, &opt, s);
    };
    // median of three timed runs, each on the restored scratch grid
    auto time_of = [&](const Candidate &c, double *ms) -> int {
        if (cudaMemcpyAsync(buf, pristine, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GBH_ECUDA;
        if (int e = run(c)) return e;
        double t[3];
        for (int r = 0; r < 3; ++r) {
            if (cudaMemcpyAsync(buf, pristine, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GBH_ECUDA;
            cudaEventRecord(e0, s);
            if (int e = run(c)) return e;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return GBH_ECUDA;
            float f = 0.f;
            cudaEventElapsedTime(&f, e0, e1);
            t[r] = f;
        }
        std::sort(t, t + 3);
        *ms = t[1];
        return GBH_OK;
    };
    int status = GBH_OK;
    double best = 1e300;
    int besti = -1;
    for (size_t i = 0; i < cands.size(); ++i) {
        double ms = 0.0;
        const int e = time_of(cands[i], &ms);
        if (e == GBH_EUNSUPPORTED) continue;    // a path that does not take the shape
        if (e != GBH_OK) { status = e; break; }
        ++out->candidates;
        if (ms < best) { best = ms; besti = (int)i; }
        if (cands[i].path == model.path && cands[i].m == model.m) out->ms_model = ms;
    }
    if (status == GBH_OK && out->ms_model == 0.0) status = time_of(model, &out->ms_model);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(buf);
    cudaFree(pristine);
    if (status != GBH_OK) return status;
    if (besti < 0) return GBH_EUNSUPPORTED;
    const Candidate &c = cands[besti];
    out->path = c.path;
    out->ms_tuned = best;
    for (size_t k = 0; k < c.m.size(); ++k) out->tile_exp[k] = c.m[k];
    out->model_path = model.path;
    for (size_t k = 0; k < model.m.size(); ++k) out->model_tile_exp[k] = model.m[k];
    // record the choice for the default path
    if (c.path == GBH_PATH_FUSED && !fused_pin_tiles(g, dtype, op, c.m.data())) return GBH_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned_path[tune_key(g, dtype, op)] = c.path;
    return GBH_OK;
}

extern "C" int gbh_autotune_reset(void)
{
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned_path.clear();
    }
    fused_forget_pins();
    return GBH_OK;
}
