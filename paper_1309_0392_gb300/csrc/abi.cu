// C ABI entry points of libgbh.so: argument validation and path dispatch.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gbh_internal.h"

namespace gbh {

static std::atomic<uint64_t> g_launches{0};

void count_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---- per-launch event timing ---------------------------------------------

namespace {
struct Pending { const char *name; cudaEvent_t a, b; double bytes; };
struct ProfStat { uint64_t n = 0; double ms = 0.0; double bytes = 0.0; };
std::mutex g_prof_mu;
std::atomic<int> g_prof_on{0};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
std::vector<std::pair<std::string, ProfStat>> g_stats;

cudaEvent_t pool_get()
{
    if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drain_pending_locked()
{
    for (auto &p : g_pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&ms, p.a, p.b);
        ProfStat *st = nullptr;
        for (auto &kv : g_stats) if (kv.first == p.name) st = &kv.second;
        if (!st) { g_stats.emplace_back(std::string(p.name), ProfStat{}); st = &g_stats.back().second; }
        st->n += 1;
        st->ms += ms;
        st->bytes += p.bytes;
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
}
}  // namespace

ProfScope::ProfScope(const char *name, cudaStream_t s, double alg_bytes)
    : name_(name), s_(s), bytes_(alg_bytes)
{
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e = pool_get();
    cudaEventRecord(e, s_);
    ev0_ = e;
}

void ProfScope::done()
{
    if (!ev0_) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e = pool_get();
    cudaEventRecord(e, s_);
    g_pending.push_back(Pending{name_, static_cast<cudaEvent_t>(ev0_), e, bytes_});
    ev0_ = nullptr;
}

int check_launch()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GBH_OK : GBH_ECUDA;
}

int num_sms()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (dev < 0 || dev >= 64) dev = 0;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 152;
        cache[dev] = v;
    }
    return cache[dev];
}

int make_geom(int d, const int32_t *levels, int elem_size, Geom *g)
{
    if (!levels || !g) return GBH_EINVAL;
    if (d < 1 || d > kMaxDim) return GBH_EINVAL;
    g->d = d;
    int64_t N = 1;
    const int64_t limit = INT64_MAX / (elem_size > 0 ? elem_size : 1);
    for (int k = 0; k < d; ++k) {
        const int l = levels[k];
        if (l < 0 || l > kMaxLevel) return GBH_ERANGE;
        g->l[k] = l;
        g->n[k] = ((int64_t)1 << l) + 1;
        g->S[k] = N;
        if (N > limit / g->n[k]) return GBH_ERANGE;
        N *= g->n[k];
    }
    g->N = N;
    g->batch = 1;
    g->total = N;
    return GBH_OK;
}

}  // namespace gbh

using namespace gbh;

extern "C" {

int gbh_num_points(int d, const int32_t *levels, int64_t *out)
{
    if (!out) return GBH_EINVAL;
    Geom g;
    if (int e = make_geom(d, levels, 1, &g)) return e;
    *out = g.N;
    return GBH_OK;
}

int gbh_tile_plan(int d, const int32_t *levels, int dtype, int op, int32_t *m_out)
{
    if (!m_out) return GBH_EINVAL;
    if (dtype != GBH_F32 && dtype != GBH_F64) return GBH_EDTYPE;
    Geom g;
    if (int e = make_geom(d, levels, dtype == GBH_F64 ? 8 : 4, &g)) return e;
    int m[kMaxDim] = {0};
    if (!fused_tiles(g, dtype, op, m)) return GBH_EUNSUPPORTED;
    for (int k = 0; k < d; ++k) m_out[k] = m[k];
    return GBH_OK;
}

int gbh_tile_candidates(int d, const int32_t *levels, int dtype, int op, int max_count, int32_t *m_out, int *count)
{
    if (!m_out || !count || max_count < 1) return GBH_EINVAL;
    if (dtype != GBH_F32 && dtype != GBH_F64) return GBH_EDTYPE;
    Geom g;
    if (int e = make_geom(d, levels, dtype == GBH_F64 ? 8 : 4, &g)) return e;
    std::vector<std::vector<int>> c;
    *count = 0;
    if (!fused_candidates(g, dtype, op, max_count, &c)) return GBH_EUNSUPPORTED;
    for (size_t i = 0; i < c.size(); ++i)
        for (int k = 0; k < d; ++k) m_out[i * d + k] = c[i][k];
    *count = (int)c.size();
    return GBH_OK;
}

int gbh_transform(void *data, int d, const int32_t *levels, int dtype, int op,
                  const gbh_options *opt, void *stream)
{
    return gbh_transform_batched(data, 1, d, levels, dtype, op, opt, stream);
}

int gbh_transform_batched(void *data, int64_t batch, int d, const int32_t *levels, int dtype,
                          int op, const gbh_options *opt, void *stream)
{
    if (dtype != GBH_F32 && dtype != GBH_F64) return GBH_EDTYPE;
    if (op != GBH_HIERARCHIZE && op != GBH_DEHIERARCHIZE && op != GBH_ADJOINT && op != GBH_DEHIERARCHIZE_ADJOINT)
        return GBH_EINVAL;
    if (!data) return GBH_EINVAL;
    const int es = dtype == GBH_F64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(data) % es) return GBH_EALIGN;
    Geom g;
    if (int e = make_geom(d, levels, es, &g)) return e;
    if (batch < 1) return GBH_EINVAL;
    if (g.N > INT64_MAX / es / batch) return GBH_ERANGE;
    g.batch = batch;
    g.total = g.N * batch;
    const int path = opt ? opt->path : GBH_PATH_AUTO;
    if (path != GBH_PATH_AUTO && path != GBH_PATH_PLAIN && path != GBH_PATH_FUSED && path != GBH_PATH_GROUPED)
        return GBH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool pairs = !(opt && opt->variant == 1);
    if (path == GBH_PATH_PLAIN) return plain_transform(data, g, dtype, op, s, opt && opt->arith == 2, pairs);
    if (path == GBH_PATH_FUSED) {
        if (!fused_supported(g, dtype, op)) return GBH_EUNSUPPORTED;
        return fused_transform(data, g, dtype, op, opt, s);
    }
    if (path == GBH_PATH_GROUPED) return grouped_transform(data, g, dtype, op, s);
    // a choice the autotuner measured for this shape, else the cost model's:
    // the fused path when it takes the shape and the grid is large enough to
    // tile, else one sweep per dimension
    const int tp = tuned_path(g, dtype, op);
    if (tp == GBH_PATH_FUSED) return fused_transform(data, g, dtype, op, opt, s);
    if (tp == GBH_PATH_GROUPED) return grouped_transform(data, g, dtype, op, s);
    if (tp != GBH_PATH_PLAIN && g.N >= 4096 && fused_preferred(g, dtype, op))
        return fused_transform(data, g, dtype, op, opt, s);
    // fp64 sweeps compute in fixed point unless native arithmetic is asked for
    // the default arithmetic (arith = 0) lets dimensions of level 1 compute natively
    return plain_transform(data, g, dtype, op, s, !(opt && opt->arith == 1), pairs, !(opt && opt->arith != 0));
}

int gbh_hierarchize(void *data, int d, const int32_t *levels, int dtype, void *stream)
{
    return gbh_transform(data, d, levels, dtype, GBH_HIERARCHIZE, nullptr, stream);
}

int gbh_dehierarchize(void *data, int d, const int32_t *levels, int dtype, void *stream)
{
    return gbh_transform(data, d, levels, dtype, GBH_DEHIERARCHIZE, nullptr, stream);
}

int gbh_hierarchize_adjoint(void *data, int d, const int32_t *levels, int dtype, void *stream)
{
    return gbh_transform(data, d, levels, dtype, GBH_ADJOINT, nullptr, stream);
}

int gbh_dehierarchize_adjoint(void *data, int d, const int32_t *levels, int dtype, void *stream)
{
    return gbh_transform(data, d, levels, dtype, GBH_DEHIERARCHIZE_ADJOINT, nullptr, stream);
}

const char *gbh_status_string(int status)
{
    switch (status) {
        case GBH_OK: return "ok";
        case GBH_EINVAL: return "invalid argument";
        case GBH_EDTYPE: return "unsupported dtype";
        case GBH_EALIGN: return "data pointer not aligned to the element size";
        case GBH_ERANGE: return "level out of range or size overflow";
        case GBH_ECUDA: return "CUDA error";
        case GBH_ETIMEOUT: return "bounded device wait expired";
        case GBH_ENOMEM: return "out of memory";
        case GBH_EUNSUPPORTED: return "unsupported option for this shape or dtype";
        default: return "unknown status";
    }
}

int gbh_launch_count(uint64_t *out)
{
    if (!out) return GBH_EINVAL;
    *out = g_launches.load(std::memory_order_relaxed);
    return GBH_OK;
}

int gbh_version(void) { return 100; }

int gbh_profile_enable(int on)
{
    g_prof_on.store(on ? 1 : 0);
    return GBH_OK;
}

int gbh_profile_read(int idx, char *name_buf, int buf_len, uint64_t *launches, double *total_ms,
                     double *total_bytes)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_pending_locked();
    if (idx < 0 || idx >= (int)g_stats.size()) return GBH_ERANGE;
    const auto &kv = g_stats[idx];
    if (name_buf && buf_len > 0) {
        std::strncpy(name_buf, kv.first.c_str(), (size_t)buf_len - 1);
        name_buf[buf_len - 1] = 0;
    }
    if (launches) *launches = kv.second.n;
    if (total_ms) *total_ms = kv.second.ms;
    if (total_bytes) *total_bytes = kv.second.bytes;
    return GBH_OK;
}

int gbh_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_pending_locked();
    g_stats.clear();
    return GBH_OK;
}

}  // extern "C"
