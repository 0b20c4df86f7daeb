/*
 * orbg_api.cpp -- the C ABI of include/orbg.h: code loading (validation,
 * GF(2) rank / null space, column packing, query-order tables, upload),
 * argument checking, host-buffer staging and kernel launches.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/orbg.h"
#include "orbg_internal.h"

struct orbg_code {
    int n, k, r, w32;
    bool has_stride = false;     /* its tables hold strided pair runs (m-segment orders) */
    uint32_t max_cap;
    int device;
    std::vector<uint8_t> H;      /* r x n as used */
    uint32_t *d_hcol = nullptr;
    OrbgRun *d_runs = nullptr;
    uint32_t *d_floor = nullptr;
    OrbgRun *d_runs_cta = nullptr;
    uint32_t *d_floor_cta = nullptr;
    uint32_t *d_trip = nullptr;
    uint32_t *d_reach = nullptr;
    uint32_t *d_reach_cta = nullptr;
    uint8_t *d_flat = nullptr;
    uint8_t *d_s3 = nullptr;
    uint32_t *d_x3off = nullptr;
    OrbgDeviceCode dev;
};

struct orbg_codeset {
    int ncodes, n_max, w32_max;
    OrbgVariants var;            /* decoder variants and the codes' sort buckets */
    int has_stride = 0;          /* a code's tables hold strided pair runs */
    int32_t *d_bucket = nullptr; /* [ncodes] sort bucket of each code (var.d_bucket) */
    uint32_t ntrip_max;
    uint32_t x3w_max;
    orbg_tuning tuning;
    std::vector<int> n_of;       /* n of each code, host copy */
    OrbgDeviceCode code0;        /* host copy of code 0's descriptor */
    uint32_t cap_min;
    int device;
    OrbgDeviceCode *d_codes = nullptr;
    /* streams of the pipelined host-buffer path (copy in, two for decodes,
     * copy out) and its host-mapped buffer for the outputs of the blocks
     * phase 2 decodes, created on first use; one pipelined call at a time */
    mutable std::mutex pipe_mu;
    mutable cudaStream_t pipe[4] = {nullptr, nullptr, nullptr, nullptr};
    mutable unsigned char *gather = nullptr;
};

namespace {

thread_local int g_last_cuda = 0;
/* smallest chunk of the pipelined host-buffer path (blocks) */
constexpr int64_t kPipeChunkMin = 65536;
/* phase-2 blocks whose outputs the pipelined path gathers in one go (more
 * and it copies every output again) */
constexpr uint32_t kGatherCap = 65536;
/* the pipelined path's answer when the layout does not suit it (nothing
 * written): the caller takes the unchunked path */
constexpr int kPipeDecline = -1;
const orbg_tuning kDefaultTuning = {8, 0, 4, 16384u, 8};

int cuda_fail(cudaError_t e)
{
    g_last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? ORBG_ENOMEM : ORBG_ECUDA;
}


/* Is p device-accessible memory the kernels may use directly? */
bool is_device_ptr(const void *p)
{
    if (!p)
        return true;
    /* an error the caller's earlier work left pending stays for the caller:
     * only the probe's own error (plain host pointers on old runtimes) is
     * cleared */
    const cudaError_t pending = cudaPeekAtLastError();
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        if (pending == cudaSuccess)
            cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

/* The library's stream-ordered memory pool on the current device.  Freed
 * memory stays reserved for the next call (release threshold unlimited):
 * from the default pool (threshold 0) it goes back to the driver at every
 * synchronisation, so a large host-buffer batch would map and unmap its
 * device buffers on every call.  orbg_pool_trim() returns it. */
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaError_t device_pool(cudaMemPool_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess)
        return e;
    uint64_t keep = UINT64_MAX;
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) !=
        cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return e;
    }
    g_pools[dev] = pool;
    *out = pool;
    return cudaSuccess;
}

/* Stream-ordered allocation from that pool; inside a stream capture, the
 * capture's own allocation node (a graph owns its allocations). */
cudaError_t alloc_async(void **p, size_t bytes, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess)
        return e;
    if (cs != cudaStreamCaptureStatusNone)
        return cudaMallocAsync(p, bytes, st);
    cudaMemPool_t pool;
    if ((e = device_pool(&pool)) != cudaSuccess)
        return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}
template <typename T>
cudaError_t alloc_async(T **p, size_t bytes, cudaStream_t st)
{
    return alloc_async((void **)p, bytes, st);
}

/* p itself, when it is page-locked host memory the device can write at
 * the same address (mapped, unified addressing); else NULL. */
template <typename T>
T *device_writable_host(T *p)
{
    const cudaError_t pending = cudaPeekAtLastError();
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        if (pending == cudaSuccess)
            cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer == (void *)p ? p : nullptr;
}

/* A device mirror of a caller buffer that lives on the host. */
struct Staged {
    void *host = nullptr;
    void *dev = nullptr;
    size_t bytes = 0;
    bool copy_in = false, copy_out = false;
};

struct Stager {
    std::vector<Staged> items;
    cudaStream_t st;
    explicit Stager(cudaStream_t s) : st(s) {}
    /* returns device pointer to use for p */
    template <typename T>
    int add(T *p, size_t bytes, bool in, bool out, T **dev_out)
    {
        if (!p || bytes == 0 || is_device_ptr(p)) {
            *dev_out = p;
            return ORBG_OK;
        }
        Staged s;
        s.host = (void *)p;
        s.bytes = bytes;
        s.copy_in = in;
        s.copy_out = out;
        cudaError_t e = alloc_async(&s.dev, bytes, st);
        if (e != cudaSuccess)
            return cuda_fail(e);
        items.push_back(s);
        if (in) {
            e = cudaMemcpyAsync(s.dev, s.host, bytes, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess)
                return cuda_fail(e);
        }
        *dev_out = (T *)s.dev;
        return ORBG_OK;
    }
    bool any() const { return !items.empty(); }
    int finish(bool ok)
    {
        int rc = ORBG_OK;
        for (auto &s : items) {
            if (ok && s.copy_out) {
                cudaError_t e = cudaMemcpyAsync(s.host, s.dev, s.bytes, cudaMemcpyDeviceToHost, st);
                if (e != cudaSuccess && rc == ORBG_OK)
                    rc = cuda_fail(e);
            }
        }
        for (auto &s : items)
            cudaFreeAsync(s.dev, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess && rc == ORBG_OK)
            rc = cuda_fail(e);
        items.clear();
        return rc;
    }
};

void free_code_device(orbg_code *c)
{
    if (c->d_hcol) cudaFree(c->d_hcol);
    if (c->d_runs) cudaFree(c->d_runs);
    if (c->d_floor) cudaFree(c->d_floor);
    if (c->d_runs_cta) cudaFree(c->d_runs_cta);
    if (c->d_floor_cta) cudaFree(c->d_floor_cta);
    if (c->d_trip) cudaFree(c->d_trip);
    if (c->d_reach) cudaFree(c->d_reach);
    if (c->d_reach_cta) cudaFree(c->d_reach_cta);
    if (c->d_flat) cudaFree(c->d_flat);
    if (c->d_s3) cudaFree(c->d_s3);
    if (c->d_x3off) cudaFree(c->d_x3off);
    c->d_s3 = nullptr;
    c->d_x3off = nullptr;
    c->d_runs_cta = nullptr;
    c->d_floor_cta = nullptr;
    c->d_trip = nullptr;
    c->d_reach = nullptr;
    c->d_reach_cta = nullptr;
    c->d_flat = nullptr;
    c->d_hcol = nullptr;
    c->d_runs = nullptr;
    c->d_floor = nullptr;
}

}  // namespace

int orbg_codeset_view(const orbg_codeset *set, OrbgSetView *out)
{
    if (!set || !out)
        return -1;
    out->d_codes = set->d_codes;
    out->code0 = set->code0;
    out->ncodes = set->ncodes;
    out->n_max = set->n_max;
    out->w32_max = set->w32_max;
    out->var = set->var;
    out->has_stride = set->has_stride;
    out->ntrip_max = set->ntrip_max;
    out->x3w_max = set->x3w_max;
    out->cap_min = set->cap_min;
    out->tuning = set->tuning;
    return 0;
}

int orbg_codeset_lengths(const orbg_codeset *set, std::vector<int> *n_of)
{
    if (!set || !n_of)
        return -1;
    *n_of = set->n_of;
    return 0;
}

int orbg_note_cuda_error(int cuda_error)
{
    return cuda_fail((cudaError_t)cuda_error);
}

extern "C" {

const char *orbg_status_string(int status)
{
    switch (status) {
    case ORBG_OK: return "ok";
    case ORBG_EINVAL: return "invalid argument";
    case ORBG_ERANK: return "matrix rank does not match n and k";
    case ORBG_ELIMIT: return "size or query cap beyond this library's limits";
    case ORBG_ENAN: return "NaN log-likelihood ratio";
    case ORBG_ENOMEM: return "out of memory";
    case ORBG_ECUDA: return "CUDA error";
    case ORBG_ETIMEOUT: return "bounded device wait ran out";
    default: return "unknown status";
    }
}

int orbg_last_cuda_error(void) { return g_last_cuda; }

int orbg_pool_trim(void)
{
    cudaMemPool_t pool;
    cudaError_t e = device_pool(&pool);
    if (e == cudaSuccess)
        e = cudaMemPoolTrimTo(pool, 0);
    return e == cudaSuccess ? ORBG_OK : cuda_fail(e);
}

int orbg_version(void) { return 200; }

int64_t orbg_query_order(int n, uint32_t count, int table, int32_t *out)
{
    return orbg_query_order_line(n, count, table, 0, 1, out);
}

namespace {

/* The first `count` patterns of table `table` of tb (orbg_query_order). */
int64_t expand_tables(const OrbgTables &tb, int n, uint32_t count, int table, int32_t *out)
{
    const std::vector<OrbgRun> &runs = table == 0 ? tb.runs : tb.runs_cta;
    const size_t stride = (size_t)n + 1;
    uint64_t total = std::min<uint64_t>(tb.patterns, count);
    if (table == 2) {
        /* the flat table: its leading patterns only */
        total = std::min<uint64_t>(total, tb.nflat);
        std::memset(out, 0, sizeof(int32_t) * stride * (size_t)total);
        for (uint64_t t = 0; t < total; t++) {
            const uint8_t *e = &tb.flat[t * 8];
            int32_t *row = out + t * stride;
            int w = 0;
            while (w < ORBG_FLAT_POS && e[w] != 0)
                w++;
            row[0] = w;
            for (int i = 0; i < w; i++)
                row[1 + i] = e[i];
        }
        return (int64_t)total;
    }
    std::memset(out, 0, sizeof(int32_t) * stride * (size_t)total);
    std::vector<int> v(64);
    for (const OrbgRun &r : runs) {
        for (int j = 0; j < r.count; j++) {
            uint64_t t = (uint64_t)r.tstart + (uint64_t)j;
            if (t > total)
                break;
            int32_t *row = out + (t - 1) * stride;
            const int w = orbg_run_pattern(r, j, tb.trip.data(), v.data());
            row[0] = w;
            for (int i = 0; i < w; i++)
                row[1 + i] = v[i];
        }
    }
    return (int64_t)total;
}

/* Checks a model given through the C ABI and fills m: anchors I_1..I_{m-1},
 * J_0..J_{m-1}, beta_1..beta_m. */
bool make_model(int n, int m, const int32_t *anchors, const int32_t *J, const int32_t *beta,
                OrbgModel *md)
{
    if (m < 1 || m > ORBG_MAX_SEG || !J || !beta || (m > 1 && !anchors))
        return false;
    md->m = m;
    md->I[0] = 0;
    md->I[m] = n;
    for (int i = 1; i < m; i++)
        md->I[i] = anchors[i - 1];
    for (int i = 0; i < m; i++) {
        md->J[i] = J[i];
        md->beta[i] = beta[i];
        if (md->I[i + 1] <= md->I[i] || beta[i] < 1 || beta[i] > ORBG_MAX_MODEL ||
            J[i] < -beta[i] || J[i] > ORBG_MAX_MODEL)
            return false;
    }
    return true;
}

}  // namespace

int64_t orbg_query_order_line(int n, uint32_t count, int table, int32_t J0, int32_t beta,
                              int32_t *out)
{
    if (n < 1 || n > ORBG_MAX_N || (count > 0 && !out) || table < 0 || table > 2 || J0 < 0 ||
        beta < 1 || J0 > ORBG_MAX_LINE || beta > ORBG_MAX_LINE)
        return ORBG_EINVAL;
    if (count == 0)
        return 0;
    OrbgTables tb;
    if (orbg_build_tables(n, count, &tb, J0, beta) != 0)
        return ORBG_ELIMIT;
    return expand_tables(tb, n, count, table, out);
}

int64_t orbg_query_order_model(int n, uint32_t count, int table, int m, const int32_t *anchors,
                               const int32_t *J, const int32_t *beta, int32_t *out)
{
    OrbgModel md;
    if (n < 1 || n > ORBG_MAX_N || (count > 0 && !out) || table < 0 || table > 2 ||
        !make_model(n, m, anchors, J, beta, &md))
        return ORBG_EINVAL;
    if (count == 0)
        return 0;
    OrbgTables tb;
    if (orbg_build_tables_model(n, count, md, &tb) != 0)
        return ORBG_ELIMIT;
    return expand_tables(tb, n, count, table, out);
}

int orbg_codeset_set_tuning(orbg_codeset *set, const orbg_tuning *t)
{
    if (!set)
        return ORBG_EINVAL;
    if (!t) {
        set->tuning = kDefaultTuning;
        return ORBG_OK;
    }
    if (t->warps_per_cta < 0 || t->warps_per_cta > 16 || t->ctas_per_sm < 0 ||
        t->ctas_per_sm > 64 || t->blocks_per_grab < 0 || t->blocks_per_grab > 1024 ||
        t->heavy_warps < 0 || t->heavy_warps > 16)
        return ORBG_EINVAL;
    orbg_tuning v = *t;
    if (!v.warps_per_cta) v.warps_per_cta = kDefaultTuning.warps_per_cta;
    if (!v.blocks_per_grab) v.blocks_per_grab = kDefaultTuning.blocks_per_grab;
    if (!v.warp_budget) v.warp_budget = kDefaultTuning.warp_budget;
    if (!v.heavy_warps) v.heavy_warps = kDefaultTuning.heavy_warps;
    set->tuning = v;
    return ORBG_OK;
}

int orbg_codeset_get_tuning(const orbg_codeset *set, orbg_tuning *t)
{
    if (!set || !t)
        return ORBG_EINVAL;
    *t = set->tuning;
    return ORBG_OK;
}

int orbg_probe_int_lanes(double *lanes_per_clk_per_sm)
{
    if (!lanes_per_clk_per_sm)
        return ORBG_EINVAL;
    int e = orbg_launch_int_probe(lanes_per_clk_per_sm);
    return e ? cuda_fail((cudaError_t)e) : ORBG_OK;
}

int orbg_probe_smem_bytes(double *bytes_per_clk_per_sm)
{
    if (!bytes_per_clk_per_sm)
        return ORBG_EINVAL;
    int e = orbg_launch_smem_probe(bytes_per_clk_per_sm);
    return e ? cuda_fail((cudaError_t)e) : ORBG_OK;
}

int orbg_load_code(const uint8_t *mat, int kind, int n, int k, uint32_t max_query_cap,
                   orbg_code **out)
{
    return orbg_load_code_line(mat, kind, n, k, max_query_cap, 0, 1, out);
}

namespace {

/* orbg_load_code for the order of model md (m-segment), or of the line
 * (J0, beta) when md is NULL. */
int load_code(const uint8_t *mat, int kind, int n, int k, uint32_t max_query_cap,
              const OrbgModel *md, int32_t J0, int32_t beta, orbg_code **out)
{
    OrbgRange range("orbg_load_code");
    if (!mat || (kind != ORBG_MAT_H && kind != ORBG_MAT_G) || n < 1 || k < 0 || k >= n)
        return ORBG_EINVAL;
    if (n > ORBG_MAX_N || n - k > ORBG_MAX_R)
        return ORBG_ELIMIT;
    uint32_t cap = max_query_cap ? max_query_cap : ORBG_DEFAULT_QUERY_CAP;
    if (cap > ORBG_MAX_QUERY_CAP)
        return ORBG_ELIMIT;
    const int r = n - k;
    const int rows = kind == ORBG_MAT_H ? r : k;
    for (size_t i = 0; i < (size_t)rows * n; i++)
        if (mat[i] > 1)
            return ORBG_EINVAL;

    orbg_code *c = new (std::nothrow) orbg_code();
    if (!c)
        return ORBG_ENOMEM;
    c->n = n;
    c->k = k;
    c->r = r;
    c->w32 = r <= 32 ? 1 : r <= 64 ? 2 : 4;
    c->max_cap = cap;
    if (kind == ORBG_MAT_H) {
        if (orbg_gf2_rank(mat, r, n) != r) {
            delete c;
            return ORBG_ERANK;
        }
        c->H.assign(mat, mat + (size_t)r * n);
    } else {
        if (k > 0 && orbg_gf2_rank(mat, k, n) != k) {
            delete c;
            return ORBG_ERANK;
        }
        int dim = 0;
        if (k == 0) {
            c->H.assign((size_t)n * n, 0);
            for (int i = 0; i < n; i++)
                c->H[(size_t)i * n + i] = 1;
            dim = n;
        } else {
            orbg_gf2_nullspace(mat, k, n, &c->H, &dim);
        }
        if (dim != r) {
            delete c;
            return ORBG_ERANK;
        }
    }
    /* columns, bit-packed: word x of column j holds rows 32x .. 32x+31 */
    std::vector<uint32_t> hcol((size_t)n * c->w32, 0);
    for (int i = 0; i < r; i++)
        for (int j = 0; j < n; j++)
            if (c->H[(size_t)i * n + j])
                hcol[(size_t)j * c->w32 + i / 32] |= 1u << (i % 32);
    OrbgTables tb;
    int trc = md ? orbg_build_tables_model(n, cap, *md, &tb)
                 : orbg_build_tables(n, cap, &tb, J0, beta);
    if (trc != 0) {
        delete c;
        return ORBG_ELIMIT;
    }
    for (const OrbgRun &run : tb.runs)
        c->has_stride |= run.kind == ORBG_RUN_STRIDE;
    for (const OrbgRun &run : tb.runs_cta)
        c->has_stride |= run.kind == ORBG_RUN_STRIDE;
    cudaError_t e;
    if ((e = cudaGetDevice(&c->device)) != cudaSuccess) {
        delete c;
        return cuda_fail(e);
    }
    /* device copies: hcol, both run tables with their floors, the triples */
    struct Up {
        void **dst;
        const void *src;
        size_t bytes;
    };
    Up ups[] = {
        {(void **)&c->d_hcol, hcol.data(), hcol.size() * sizeof(uint32_t)},
        {(void **)&c->d_runs, tb.runs.data(), tb.runs.size() * sizeof(OrbgRun)},
        {(void **)&c->d_floor, tb.group_floor.data(), tb.group_floor.size() * sizeof(uint32_t)},
        {(void **)&c->d_runs_cta, tb.runs_cta.data(), tb.runs_cta.size() * sizeof(OrbgRun)},
        {(void **)&c->d_floor_cta, tb.group_floor_cta.data(),
         tb.group_floor_cta.size() * sizeof(uint32_t)},
        {(void **)&c->d_trip, tb.trip.data(), tb.trip.size() * 4},
        {(void **)&c->d_reach, tb.reach.data(), tb.reach.size() * 4},
        {(void **)&c->d_reach_cta, tb.reach_cta.data(), tb.reach_cta.size() * 4},
        {(void **)&c->d_flat, tb.flat.data(), tb.flat.size()},
        {(void **)&c->d_s3, tb.s3_cta.data(), tb.s3_cta.size()},
        {(void **)&c->d_x3off, tb.x3off.data(), tb.x3off.size() * 4},
    };
    for (const Up &u : ups) {
        const size_t bytes = std::max<size_t>(u.bytes, 4);
        if ((e = cudaMalloc(u.dst, bytes)) != cudaSuccess ||
            (u.bytes && (e = cudaMemcpy(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice)) !=
                            cudaSuccess)) {
            free_code_device(c);
            delete c;
            return cuda_fail(e);
        }
    }
    c->dev.hcol = c->d_hcol;
    c->dev.warp.runs = c->d_runs;
    c->dev.warp.group_floor = c->d_floor;
    c->dev.warp.nruns = (uint32_t)tb.runs.size();
    c->dev.warp.ngroups = (uint32_t)tb.group_floor.size();
    c->dev.warp.group_reach = c->d_reach;
    c->dev.warp.flat_group = tb.flat_group;
    c->dev.cta.runs = c->d_runs_cta;
    c->dev.cta.group_floor = c->d_floor_cta;
    c->dev.cta.nruns = (uint32_t)tb.runs_cta.size();
    c->dev.cta.ngroups = (uint32_t)tb.group_floor_cta.size();
    c->dev.cta.group_reach = c->d_reach_cta;
    c->dev.cta.group_s3 = c->d_s3;
    c->dev.x3off = c->d_x3off;
    c->dev.s3max = tb.s3max;
    c->dev.exact16 = r <= 16 ? 1 : 0;
    c->dev.x3w = tb.x3off[std::min(ORBG_X3_WARP_S3, tb.s3max) + 1];
    c->dev.cta.flat_group = tb.flat_group_cta;
    c->dev.flat = reinterpret_cast<const uint32_t *>(c->d_flat);
    c->dev.nflat = tb.nflat;
    c->dev.trip = c->d_trip;
    c->dev.ntrip = (uint32_t)tb.trip.size();
    c->dev.max_cap = cap;
    c->dev.n = n;
    c->dev.r = r;
    c->dev.w32 = c->w32;
    *out = c;
    return ORBG_OK;
}

}  // namespace

int orbg_load_code_line(const uint8_t *mat, int kind, int n, int k, uint32_t max_query_cap,
                        int32_t J0, int32_t beta, orbg_code **out)
{
    if (!out)
        return ORBG_EINVAL;
    *out = nullptr;
    if (J0 < 0 || beta < 1 || J0 > ORBG_MAX_LINE || beta > ORBG_MAX_LINE)
        return ORBG_EINVAL;
    return load_code(mat, kind, n, k, max_query_cap, nullptr, J0, beta, out);
}

int orbg_load_code_model(const uint8_t *mat, int kind, int n, int k, uint32_t max_query_cap,
                         int m, const int32_t *anchors, const int32_t *J, const int32_t *beta,
                         orbg_code **out)
{
    if (!out)
        return ORBG_EINVAL;
    *out = nullptr;
    OrbgModel md;
    if (n < 1 || !make_model(n, m, anchors, J, beta, &md))
        return ORBG_EINVAL;
    return load_code(mat, kind, n, k, max_query_cap, &md, 0, 1, out);
}

int orbg_free_code(orbg_code *code)
{
    if (!code)
        return ORBG_OK;
    free_code_device(code);
    delete code;
    return ORBG_OK;
}

int orbg_code_info(const orbg_code *code, int *n, int *k, uint32_t *max_query_cap,
                   uint8_t *H_out)
{
    if (!code)
        return ORBG_EINVAL;
    if (n) *n = code->n;
    if (k) *k = code->k;
    if (max_query_cap) *max_query_cap = code->max_cap;
    if (H_out) std::memcpy(H_out, code->H.data(), code->H.size());
    return ORBG_OK;
}

int orbg_decode(const orbg_code *code, const float *llr, int64_t B, uint32_t query_cap,
                uint8_t *codeword, uint32_t *queries, uint8_t *abandoned, void *cuda_stream)
{
    OrbgRange range("orbg_decode");
    if (!code || B < 0)
        return ORBG_EINVAL;
    if (query_cap < 1)
        return ORBG_EINVAL;
    if (query_cap > code->max_cap)
        return ORBG_ELIMIT;
    if (B == 0)
        return ORBG_OK;
    if (!llr || !codeword || !queries || !abandoned)
        return ORBG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t nb = (size_t)B * code->n;
    Stager sg(st);
    const float *d_llr;
    uint8_t *d_cw, *d_ab;
    uint32_t *d_q;
    int rc;
    if ((rc = sg.add(llr, nb * sizeof(float), true, false, &d_llr)) ||
        (rc = sg.add(codeword, nb, false, true, &d_cw)) ||
        (rc = sg.add(queries, (size_t)B * sizeof(uint32_t), false, true, &d_q)) ||
        (rc = sg.add(abandoned, (size_t)B, false, true, &d_ab))) {
        sg.finish(false);
        return rc;
    }
    int e = orbg_launch_plain(code->dev, d_llr, B, query_cap, d_cw, d_q, d_ab, st);
    if (e != 0) {
        sg.finish(false);
        return cuda_fail((cudaError_t)e);
    }
    if (!sg.any())
        return ORBG_OK;
    rc = sg.finish(true);
    if (rc)
        return rc;
    if (!is_device_ptr(abandoned) && std::memchr(abandoned, ORBG_BLOCK_NAN, (size_t)B))
        return ORBG_ENAN;
    return ORBG_OK;
}

int orbg_codeset_create(const orbg_code *const *codes, int ncodes, orbg_codeset **out)
{
    if (!out)
        return ORBG_EINVAL;
    *out = nullptr;
    if (!codes || ncodes < 1 || ncodes > ORBG_MAX_CODES)
        return ORBG_EINVAL;
    std::vector<OrbgDeviceCode> descs((size_t)ncodes);
    orbg_codeset *s = new (std::nothrow) orbg_codeset();
    if (!s)
        return ORBG_ENOMEM;
    s->ncodes = ncodes;
    s->n_max = 0;
    s->w32_max = 1;
    s->cap_min = 0xFFFFFFFFu;
    s->ntrip_max = 0;
    s->x3w_max = 0;
    s->tuning = kDefaultTuning;
    for (int i = 0; i < ncodes; i++) {
        if (!codes[i]) {
            delete s;
            return ORBG_EINVAL;
        }
        descs[i] = codes[i]->dev;
        if (i == 0)
            s->code0 = codes[i]->dev;
        s->n_of.push_back(codes[i]->n);
        s->n_max = std::max(s->n_max, codes[i]->n);
        s->w32_max = std::max(s->w32_max, codes[i]->w32);
        s->cap_min = std::min(s->cap_min, codes[i]->max_cap);
        s->ntrip_max = std::max(s->ntrip_max, codes[i]->dev.ntrip);
        s->x3w_max = std::max(s->x3w_max, codes[i]->dev.x3w);
        s->has_stride |= codes[i]->has_stride ? 1 : 0;
    }
    /* the decoder variants the kernels specialise on: keys per lane from n
     * (n <= 32, 64, 128, 256: 1, 2, 4, 8) and the syndrome words (1, 2, or
     * 4 for 3-4); the codes in order of (variant, id) number the sort
     * buckets, so each variant's codes hold consecutive buckets */
    std::vector<int32_t> bucket((size_t)ncodes);
    {
        std::vector<int> key((size_t)ncodes), ord((size_t)ncodes);
        for (int i = 0; i < ncodes; i++) {
            const int n = codes[i]->n, w = codes[i]->w32;
            key[i] = (n <= 32 ? 1 : n <= 64 ? 2 : n <= 128 ? 4 : 8) * 8 +
                     (w <= 1 ? 1 : w == 2 ? 2 : 4);
            ord[i] = i;
        }
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return key[x] < key[y]; });
        OrbgVariants &v = s->var;
        v = OrbgVariants{};
        for (int j = 0; j < ncodes; j++) {
            bucket[ord[j]] = j;
            if (j == 0 || key[ord[j]] != key[ord[j - 1]]) {
                v.k[v.n] = key[ord[j]] / 8;
                v.w[v.n] = key[ord[j]] % 8;
                v.blo[v.n] = j;
                v.n++;
            }
            v.bhi[v.n - 1] = j + 1;
        }
        v.bhi[v.n - 1] = ncodes + 1; /* ids outside the set go with the last variant */
    }
    cudaError_t e;
    if ((e = cudaGetDevice(&s->device)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_codes, descs.size() * sizeof(OrbgDeviceCode))) != cudaSuccess ||
        (e = cudaMemcpy(s->d_codes, descs.data(), descs.size() * sizeof(OrbgDeviceCode),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_bucket, bucket.size() * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMemcpy(s->d_bucket, bucket.data(), bucket.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice)) != cudaSuccess) {
        if (s->d_codes) cudaFree(s->d_codes);
        if (s->d_bucket) cudaFree(s->d_bucket);
        delete s;
        return cuda_fail(e);
    }
    s->var.d_bucket = s->d_bucket;
    *out = s;
    return ORBG_OK;
}

int orbg_codeset_free(orbg_codeset *set)
{
    if (!set)
        return ORBG_OK;
    if (set->d_codes)
        cudaFree(set->d_codes);
    if (set->d_bucket)
        cudaFree(set->d_bucket);
    for (cudaStream_t s : set->pipe)
        if (s)
            cudaStreamDestroy(s);
    if (set->gather)
        cudaFreeHost(set->gather);
    delete set;
    return ORBG_OK;
}

namespace {

/*
 * Host buffers and a large batch: the batch is cut into chunks of
 * consecutive blocks.  Each chunk's host-to-device copy (one stream) is
 * followed by phase 1 over its blocks, on two decode streams taken in turn
 * (with a queue slot each in the scratch), so chunk i's copy in overlaps
 * chunk i-1's decode, and the next chunk's launch fills the SMs that the
 * end of the previous one leaves idle; each chunk's results go back (a
 * fourth stream) while later chunks decode.  The blocks every chunk leaves
 * open go to one list, which a single phase-2 launch searches after the
 * last chunk (one tail for the batch, not one per chunk).  A gather then
 * writes their outputs over what the chunk copies brought: straight into
 * the caller's buffers when they are page-locked and mapped (after those
 * copies have landed), else into a host-mapped staging buffer that the
 * host spreads once everything has finished.  Each block is decoded
 * exactly as by an unchunked call.
 *
 * The layout is dense (one code, no offsets) or given by host offsets that
 * place every block at or after the end of the one before, in both
 * buffers, so that each chunk is one contiguous range of each.  The host
 * checks this chunk by chunk, before the chunk's copy and launch, so the
 * check of chunk i + 1 runs while the device works on chunk i.  When a
 * chunk fails it (blocks out of order, a code id outside the set) nothing
 * has been written to the outputs yet, and the call returns kPipeDecline
 * for the unchunked path (which rejects invalid ids).  Synchronises `st`.
 */
int decode_batched_pipelined(const orbg_codeset *set, const int32_t *code_id,
                             const int64_t *llr_offset, const float *llr, int64_t B,
                             uint32_t query_cap, uint8_t *codeword, const int64_t *cw_offset,
                             uint32_t *queries, uint8_t *abandoned, cudaStream_t st)
{
    if (!llr_offset && code_id)
        return kPipeDecline; /* a dense layout holds one code */
    const int64_t n0 = set->n_of[0];
    /* the buffers' extents if the layout is ordered: the last block ends them */
    int64_t n_llr = B * n0, n_cw = B * n0;
    if (llr_offset) {
        const int32_t c = code_id ? code_id[B - 1] : 0;
        if (c < 0 || c >= set->ncodes || llr_offset[0] < 0 || cw_offset[0] < 0 ||
            llr_offset[B - 1] > (INT64_MAX >> 2) || cw_offset[B - 1] > (INT64_MAX >> 2))
            return kPipeDecline;
        n_llr = llr_offset[B - 1] + set->n_of[c];
        n_cw = cw_offset[B - 1] + set->n_of[c];
    }
    /* first element of block b in each buffer; block B marks the end */
    auto llr_at = [&](int64_t b) -> int64_t {
        return b >= B ? n_llr : llr_offset ? llr_offset[b] : b * n0;
    };
    auto cw_at = [&](int64_t b) -> int64_t {
        return b >= B ? n_cw : cw_offset ? cw_offset[b] : b * n0;
    };
    /* blocks [b0, b1) have codes of the set, each ends at or before the
     * start of the next (the first starts at or after 0, checked above) and
     * within the extents taken from the last block (a chunk whose copy would
     * reach past them is refused before it is made) */
    auto ordered = [&](int64_t b0, int64_t b1) -> bool {
        if (!llr_offset)
            return true;
        for (int64_t b = b0; b < b1; b++) {
            const int32_t c = code_id ? code_id[b] : 0;
            if (c < 0 || c >= set->ncodes)
                return false;
            const int64_t n = set->n_of[c];
            if (llr_at(b + 1) < llr_offset[b] + n || cw_at(b + 1) < cw_offset[b] + n ||
                llr_at(b + 1) > n_llr || cw_at(b + 1) > n_cw)
                return false;
        }
        return true;
    };
    std::lock_guard<std::mutex> lk(set->pipe_mu);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 4 && e == cudaSuccess; i++)
        if (!set->pipe[i])
            e = cudaStreamCreateWithFlags(&set->pipe[i], cudaStreamNonBlocking);
    if (e == cudaSuccess && !set->gather)
        e = cudaHostAlloc((void **)&set->gather, orbg_gather_bytes(kGatherCap, set->n_max),
                          cudaHostAllocMapped);
    unsigned char *d_gather = nullptr;
    if (e == cudaSuccess)
        e = cudaHostGetDevicePointer((void **)&d_gather, set->gather, 0);
    if (e != cudaSuccess)
        return cuda_fail(e);
    cudaStream_t s_in = set->pipe[0], s_dec = set->pipe[1], s_out = set->pipe[2],
                 s_dec1 = set->pipe[3];
    /* the caller's output buffers, when the gather can write them in place */
    uint8_t *to_cw = device_writable_host(codeword);
    uint32_t *to_q = device_writable_host(queries);
    uint8_t *to_ab = device_writable_host(abandoned);
    const bool in_place = to_cw && to_q && to_ab;
    /* chunk bounds: up to eight equal chunks, the first of them cut into a
     * quarter and three quarters when it is large enough, so that decoding
     * starts after a shorter first copy */
    std::vector<int64_t> cut;
    {
        const int64_t nch = std::min<int64_t>(8, B / kPipeChunkMin);
        const int64_t per = (B + nch - 1) / nch;
        cut.push_back(0);
        for (int64_t i = 0; i < nch; i++) {
            const int64_t b0 = i * per, b1 = std::min(B, b0 + per);
            if (b1 <= b0)
                break;
            if (i == 0 && per / 4 >= kPipeChunkMin / 4)
                cut.push_back(b0 + per / 4);
            cut.push_back(b1);
        }
    }
    const int64_t nch = (int64_t)cut.size() - 1;
    float *d_llr = nullptr;
    uint8_t *d_cw = nullptr, *d_ab = nullptr;
    uint32_t *d_q = nullptr;
    int32_t *d_cid = nullptr;
    int64_t *d_lo = nullptr, *d_co = nullptr;
    unsigned long long *scratch = nullptr;
    std::vector<cudaEvent_t> ev;
    auto event = [&](cudaEvent_t *out) -> cudaError_t {
        cudaError_t r = cudaEventCreateWithFlags(out, cudaEventDisableTiming);
        if (r == cudaSuccess)
            ev.push_back(*out);
        return r;
    };
    cudaEvent_t start = nullptr;
    if ((e = alloc_async(&d_llr, (size_t)n_llr * sizeof(float), st)) != cudaSuccess ||
        (e = alloc_async(&d_cw, (size_t)n_cw, st)) != cudaSuccess ||
        (e = alloc_async(&d_q, (size_t)B * sizeof(uint32_t), st)) != cudaSuccess ||
        (e = alloc_async(&d_ab, (size_t)B, st)) != cudaSuccess ||
        (e = alloc_async(&scratch, orbg_batched_scratch_bytes(B, set->ncodes), st)) !=
            cudaSuccess ||
        (code_id && (e = alloc_async(&d_cid, (size_t)B * sizeof(int32_t), st)) !=
                        cudaSuccess) ||
        (llr_offset && (e = alloc_async(&d_lo, (size_t)B * sizeof(int64_t), st)) !=
                           cudaSuccess) ||
        (cw_offset && (e = alloc_async(&d_co, (size_t)B * sizeof(int64_t), st)) !=
                          cudaSuccess) ||
        /* the whole scratch cleared once, before either decode stream
         * starts; each chunk then resets only its own slot */
        (e = cudaMemsetAsync(scratch, 0, orbg_scratch_layout(scratch, B, set->ncodes).zero_bytes,
                             st)) != cudaSuccess ||
        (e = event(&start)) != cudaSuccess || (e = cudaEventRecord(start, st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s_in, start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s_dec, start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s_dec1, start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s_out, start, 0)) != cudaSuccess) {
        /* fall through to clean-up */
    }
    /* the per-block layout arrays go first, whole (12 bytes a block); the
     * kernels read a chunk's entries only after the host checked them */
    if (e == cudaSuccess && code_id)
        e = cudaMemcpyAsync(d_cid, code_id, (size_t)B * sizeof(int32_t), cudaMemcpyHostToDevice,
                            s_in);
    if (e == cudaSuccess && llr_offset)
        e = cudaMemcpyAsync(d_lo, llr_offset, (size_t)B * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess && cw_offset)
        e = cudaMemcpyAsync(d_co, cw_offset, (size_t)B * sizeof(int64_t), cudaMemcpyHostToDevice,
                            s_in);
    const orbg_tuning &t = set->tuning;
    int le = 0;
    OrbgBatchedArgs a{};
    a.d_codes = set->d_codes;
    a.code0 = &set->code0;
    a.ncodes = set->ncodes;
    a.n_max = set->n_max;
    a.w32_max = set->w32_max;
    a.var = set->var;
    a.has_stride = set->has_stride;
    a.cap = query_cap;
    a.budget = t.warp_budget < query_cap ? t.warp_budget : query_cap;
    a.scratch = scratch;
    a.warps_per_cta = t.warps_per_cta;
    a.ctas_per_sm = t.ctas_per_sm;
    a.grab = t.blocks_per_grab;
    a.heavy_warps = t.heavy_warps;
    a.ntrip_max = set->ntrip_max;
    a.x3w_max = set->x3w_max;
    a.scratch_B = B;
    bool declined = false;
    std::vector<cudaEvent_t> chunk_done;
    for (int64_t i = 0; i < nch && e == cudaSuccess && le == 0; i++) {
        const int64_t b0 = cut[(size_t)i], b1 = cut[(size_t)i + 1];
        if (b1 <= b0)
            break;
        if (!ordered(b0, b1)) {
            declined = true;
            break;
        }
        const int64_t l0 = llr_at(b0), l1 = llr_at(b1), c0 = cw_at(b0);
        cudaStream_t sd = (i & 1) ? s_dec1 : s_dec;
        cudaEvent_t in_done = nullptr, dec_done = nullptr;
        if ((e = event(&in_done)) != cudaSuccess || (e = event(&dec_done)) != cudaSuccess)
            break;
        if ((e = cudaMemcpyAsync(d_llr + l0, llr + l0, (size_t)(l1 - l0) * sizeof(float),
                                 cudaMemcpyHostToDevice, s_in)) != cudaSuccess ||
            (e = cudaEventRecord(in_done, s_in)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(sd, in_done, 0)) != cudaSuccess)
            break;
        /* phase 1 of this chunk; dense chunks index from their own first
         * block, offsets are absolute in the whole buffers */
        a.code_id = d_cid ? d_cid + b0 : nullptr;
        a.llr_off = d_lo ? d_lo + b0 : nullptr;
        a.cw_off = d_co ? d_co + b0 : nullptr;
        a.llr = d_lo ? d_llr : d_llr + l0;
        a.cw = d_co ? d_cw : d_cw + c0;
        a.B = b1 - b0;
        a.q = d_q + b0;
        a.ab = d_ab + b0;
        a.stage = 1;
        a.slot = (int)(i & 1);
        a.first_chunk = 0;
        a.scratch_base = b0;
        a.stream = sd;
        if ((le = orbg_launch_batched(a)) != 0)
            break;
        if ((e = cudaEventRecord(dec_done, sd)) != cudaSuccess)
            break;
        chunk_done.push_back(dec_done);
    }
    const bool go = e == cudaSuccess && le == 0 && !declined;
    /* every chunk's results out as soon as its phase 1 is done */
    for (size_t i = 0; go && e == cudaSuccess && i < chunk_done.size(); i++) {
        const int64_t b0 = cut[i], b1 = cut[i + 1];
        const int64_t c0 = cw_at(b0), c1 = cw_at(b1);
        if ((e = cudaStreamWaitEvent(s_out, chunk_done[i], 0)) != cudaSuccess ||
            (c1 > c0 && (e = cudaMemcpyAsync(codeword + c0, d_cw + c0, (size_t)(c1 - c0),
                                             cudaMemcpyDeviceToHost, s_out)) != cudaSuccess) ||
            (e = cudaMemcpyAsync(queries + b0, d_q + b0, (size_t)(b1 - b0) * sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, s_out)) != cudaSuccess ||
            (e = cudaMemcpyAsync(abandoned + b0, d_ab + b0, (size_t)(b1 - b0),
                                 cudaMemcpyDeviceToHost, s_out)) != cudaSuccess)
            break;
    }
    /* phase 2 once, over the whole batch, after both decode streams; then
     * its blocks' outputs gathered (in place: after the chunk copies) */
    cudaEvent_t dec1_done = nullptr, out_done = nullptr;
    if (go && e == cudaSuccess &&
        ((e = event(&dec1_done)) != cudaSuccess ||
         (e = cudaEventRecord(dec1_done, s_dec1)) != cudaSuccess ||
         (e = cudaStreamWaitEvent(s_dec, dec1_done, 0)) != cudaSuccess)) {
        /* fall through to the join */
    }
    if (go && e == cudaSuccess) {
        a.stream = s_dec;
        a.code_id = d_cid;
        a.llr_off = d_lo;
        a.cw_off = d_co;
        a.llr = d_llr;
        a.cw = d_cw;
        a.B = B;
        a.q = d_q;
        a.ab = d_ab;
        a.stage = 2;
        a.first_chunk = 0;
        a.scratch_base = 0;
        le = orbg_launch_batched(a);
        if (le == 0 && in_place &&
            ((e = event(&out_done)) != cudaSuccess ||
             (e = cudaEventRecord(out_done, s_out)) != cudaSuccess ||
             (e = cudaStreamWaitEvent(s_dec, out_done, 0)) != cudaSuccess)) {
            /* fall through to the join */
        } else if (le == 0) {
            le = orbg_launch_heavy_gather(set->d_codes, d_cid, (int)n0, d_co, d_cw, d_q, d_ab,
                                          orbg_scratch_layout(scratch, B, set->ncodes), d_gather,
                                          kGatherCap, set->n_max, in_place ? to_cw : nullptr,
                                          to_q, to_ab, s_dec);
        }
    }
    /* join: the caller's stream waits for all four */
    auto join = [&]() -> cudaError_t {
        cudaError_t je = cudaSuccess;
        cudaEvent_t done = nullptr;
        for (cudaStream_t sx : {s_in, s_dec, s_dec1, s_out}) {
            if (je == cudaSuccess && (je = event(&done)) == cudaSuccess &&
                (je = cudaEventRecord(done, sx)) == cudaSuccess)
                je = cudaStreamWaitEvent(st, done, 0);
        }
        if (je == cudaSuccess)
            je = cudaStreamSynchronize(st);
        return je;
    };
    cudaError_t je = join();
    /* more phase-2 blocks than the staging buffer holds: copy every output
     * again */
    int rc = ORBG_OK;
    const uint64_t nheavy = *(volatile uint64_t *)set->gather;
    if (go && le == 0 && e == cudaSuccess && je == cudaSuccess && !in_place &&
        nheavy > kGatherCap) {
        if ((e = cudaMemcpyAsync(codeword, d_cw, (size_t)n_cw, cudaMemcpyDeviceToHost, st)) ==
                cudaSuccess &&
            (e = cudaMemcpyAsync(queries, d_q, (size_t)B * sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, st)) == cudaSuccess &&
            (e = cudaMemcpyAsync(abandoned, d_ab, (size_t)B, cudaMemcpyDeviceToHost, st)) ==
                cudaSuccess)
            e = cudaStreamSynchronize(st);
    }
    for (void *ptr : {(void *)d_llr, (void *)d_cw, (void *)d_q, (void *)d_ab, (void *)scratch,
                      (void *)d_cid, (void *)d_lo, (void *)d_co})
        if (ptr)
            cudaFreeAsync(ptr, st);
    for (cudaEvent_t x : ev)
        cudaEventDestroy(x);
    if (e != cudaSuccess)
        return cuda_fail(e);
    if (le != 0)
        return cuda_fail((cudaError_t)le);
    if (je != cudaSuccess)
        return cuda_fail(je);
    if (declined)
        return kPipeDecline;
    if (!in_place && nheavy <= kGatherCap) {
        /* the phase-2 blocks' outputs over what the chunk copies brought */
        const unsigned char *g = set->gather;
        const uint32_t *bq = (const uint32_t *)(g + 16);
        const uint8_t *flag = g + 16 + 8 * (size_t)kGatherCap;
        const uint8_t *cwg = g + orbg_gather_cw_at(kGatherCap);
        for (uint64_t h = 0; h < nheavy; h++) {
            const int64_t b = bq[2 * h];
            if (b >= B)
                return cuda_fail(cudaErrorUnknown); /* not a block of this call */
            std::memcpy(codeword + cw_at(b), cwg + h * (size_t)set->n_max,
                        (size_t)set->n_of[code_id ? code_id[b] : 0]);
            queries[b] = bq[2 * h + 1];
            abandoned[b] = flag[h];
        }
    }
    if (std::memchr(abandoned, ORBG_BLOCK_NAN, (size_t)B))
        rc = ORBG_ENAN;
    return rc;
}

}  // namespace

int orbg_decode_batched(const orbg_codeset *set, const int32_t *code_id,
                        const int64_t *llr_offset, const float *llr, int64_t B,
                        uint32_t query_cap, uint8_t *codeword, const int64_t *cw_offset,
                        uint32_t *queries, uint8_t *abandoned, void *cuda_stream)
{
    OrbgRange range("orbg_decode_batched");
    if (!set || B < 0 || query_cap < 1)
        return ORBG_EINVAL;
    if (query_cap > set->cap_min || B >= ((int64_t)1 << 32))
        return ORBG_ELIMIT;
    if (B == 0)
        return ORBG_OK;
    if (!llr || !codeword || !queries || !abandoned)
        return ORBG_EINVAL;
    if ((llr_offset == nullptr) != (cw_offset == nullptr))
        return ORBG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    /* large batches on host buffers: chunked, copies overlapping decodes,
     * when every layout array is on the host and places blocks in order */
    if (B >= 2 * kPipeChunkMin && !is_device_ptr(llr) && !is_device_ptr(codeword) &&
        !is_device_ptr(queries) && !is_device_ptr(abandoned) &&
        (!code_id || !is_device_ptr(code_id)) && (!llr_offset || !is_device_ptr(llr_offset)) &&
        (!cw_offset || !is_device_ptr(cw_offset))) {
        const int rc = decode_batched_pipelined(set, code_id, llr_offset, llr, B, query_cap,
                                                codeword, cw_offset, queries, abandoned, st);
        if (rc != kPipeDecline)
            return rc;
    }
    /* element counts: dense layout, or as far as the largest offset reaches */
    size_t n_llr, n_cw;
    if (!llr_offset) {
        n_llr = n_cw = (size_t)B * set->n_of[0];
    } else {
        if (!is_device_ptr(llr_offset) || !is_device_ptr(cw_offset) ||
            (code_id && !is_device_ptr(code_id))) {
            /* host-side layout arrays: find extents for staging */
            if (is_device_ptr(llr_offset) || is_device_ptr(cw_offset) ||
                (code_id && is_device_ptr(code_id)))
                return ORBG_EINVAL;
            int64_t hi_l = 0, hi_c = 0;
            for (int64_t b = 0; b < B; b++) {
                int cid = code_id ? code_id[b] : 0;
                if (cid < 0 || cid >= set->ncodes || llr_offset[b] < 0 || cw_offset[b] < 0)
                    return ORBG_EINVAL;
                hi_l = std::max(hi_l, llr_offset[b] + set->n_of[cid]);
                hi_c = std::max(hi_c, cw_offset[b] + set->n_of[cid]);
            }
            n_llr = (size_t)hi_l;
            n_cw = (size_t)hi_c;
        } else {
            if (!is_device_ptr(llr) || !is_device_ptr(codeword))
                return ORBG_EINVAL; /* device layout arrays need device data */
            n_llr = n_cw = 0;
        }
    }
    Stager sg(st);
    const float *d_llr;
    uint8_t *d_cw, *d_ab;
    uint32_t *d_q;
    const int32_t *d_cid;
    const int64_t *d_lo, *d_co;
    int rc;
    if ((rc = sg.add(code_id, code_id ? (size_t)B * sizeof(int32_t) : 0, true, false, &d_cid)) ||
        (rc = sg.add(llr_offset, llr_offset ? (size_t)B * sizeof(int64_t) : 0, true, false,
                     &d_lo)) ||
        (rc = sg.add(cw_offset, cw_offset ? (size_t)B * sizeof(int64_t) : 0, true, false,
                     &d_co)) ||
        (rc = sg.add(llr, n_llr * sizeof(float), true, false, &d_llr)) ||
        (rc = sg.add(codeword, n_cw, false, true, &d_cw)) ||
        (rc = sg.add(queries, (size_t)B * sizeof(uint32_t), false, true, &d_q)) ||
        (rc = sg.add(abandoned, (size_t)B, false, true, &d_ab))) {
        sg.finish(false);
        return rc;
    }
    unsigned long long *scratch = nullptr;
    cudaError_t e = alloc_async(&scratch, orbg_batched_scratch_bytes(B, set->ncodes), st);
    if (e != cudaSuccess) {
        sg.finish(false);
        return cuda_fail(e);
    }
    const orbg_tuning &t = set->tuning;
    const uint32_t budget = t.warp_budget < query_cap ? t.warp_budget : query_cap;
    OrbgBatchedArgs a{};
    a.d_codes = set->d_codes;
    a.code0 = &set->code0;
    a.ncodes = set->ncodes;
    a.n_max = set->n_max;
    a.w32_max = set->w32_max;
    a.var = set->var;
    a.has_stride = set->has_stride;
    a.code_id = d_cid;
    a.llr_off = d_lo;
    a.llr = d_llr;
    a.B = B;
    a.cap = query_cap;
    a.budget = budget;
    a.cw = d_cw;
    a.cw_off = d_co;
    a.q = d_q;
    a.ab = d_ab;
    a.scratch = scratch;
    a.warps_per_cta = t.warps_per_cta;
    a.ctas_per_sm = t.ctas_per_sm;
    a.grab = t.blocks_per_grab;
    a.heavy_warps = t.heavy_warps;
    a.ntrip_max = set->ntrip_max;
    a.x3w_max = set->x3w_max;
    a.stream = st;
    int le = orbg_launch_batched(a);
    cudaFreeAsync(scratch, st);
    if (le != 0) {
        sg.finish(false);
        return cuda_fail((cudaError_t)le);
    }
    if (!sg.any())
        return ORBG_OK;
    rc = sg.finish(true);
    if (rc)
        return rc;
    if (!is_device_ptr(abandoned) && std::memchr(abandoned, ORBG_BLOCK_NAN, (size_t)B))
        return ORBG_ENAN;
    return ORBG_OK;
}

int orbg_codeset_autotune(orbg_codeset *set, const int32_t *code_id, const int64_t *llr_offset,
                          const float *llr, int64_t B, uint32_t query_cap, uint8_t *codeword,
                          const int64_t *cw_offset, uint32_t *queries, uint8_t *abandoned,
                          int reps, void *cuda_stream, orbg_tuning *best)
{
    OrbgRange range("orbg_codeset_autotune");
    if (!set || B < 1 || reps < 0 || reps > 64)
        return ORBG_EINVAL;
    if (!is_device_ptr(llr) || !is_device_ptr(codeword) || !is_device_ptr(queries) ||
        !is_device_ptr(abandoned))
        return ORBG_EINVAL;
    const int r = reps ? reps : 3;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce;
    if ((ce = cudaEventCreate(&e0)) != cudaSuccess || (ce = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(ce);
    }
    /* median time of r runs of one tuning, ms; negative status on error */
    auto trial = [&](const orbg_tuning &t, float *ms) -> int {
        int rc = orbg_codeset_set_tuning(set, &t);
        if (rc) return rc;
        rc = orbg_decode_batched(set, code_id, llr_offset, llr, B, query_cap, codeword,
                                 cw_offset, queries, abandoned, cuda_stream); /* warm-up */
        if (rc) return rc;
        std::vector<float> v;
        for (int i = 0; i < r; i++) {
            cudaEventRecord(e0, st);
            rc = orbg_decode_batched(set, code_id, llr_offset, llr, B, query_cap, codeword,
                                     cw_offset, queries, abandoned, cuda_stream);
            if (rc) return rc;
            cudaEventRecord(e1, st);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) return cuda_fail(e);
            float x = 0;
            cudaEventElapsedTime(&x, e0, e1);
            v.push_back(x);
        }
        std::sort(v.begin(), v.end());
        *ms = v[v.size() / 2];
        return ORBG_OK;
    };
    orbg_tuning cur = set->tuning;
    float cur_ms = 0;
    int rc = trial(cur, &cur_ms);
    const uint32_t budgets[] = {256u, 1024u, 4096u, 16384u, 65536u};
    const int heavy[] = {4, 8, 16};
    const int grabs[] = {1, 4, 8, 32};
    const int wpcs[] = {4, 8};
    const int cps[] = {0, 2, 3};
    /* coordinate descent, repeated while a pass still changes something
     * (the budget and the phase-2 width interact: one pass can stop at a
     * budget that only suited the starting width) */
    for (int pass = 0; pass < 3 && rc == ORBG_OK; pass++) {
      const orbg_tuning before = cur;
      for (int knob = 0; knob < 5 && rc == ORBG_OK; knob++) {
        const int count = knob == 0 ? 5 : knob == 1 ? 3 : knob == 2 ? 4 : knob == 3 ? 2 : 3;
        for (int i = 0; i < count && rc == ORBG_OK; i++) {
            orbg_tuning t = cur;
            switch (knob) {
            case 0: t.warp_budget = budgets[i]; break;
            case 1: t.heavy_warps = heavy[i]; break;
            case 2: t.blocks_per_grab = grabs[i]; break;
            case 3: t.warps_per_cta = wpcs[i]; break;
            default: t.ctas_per_sm = cps[i]; break;
            }
            if (std::memcmp(&t, &cur, sizeof(t)) == 0)
                continue;
            float ms = 0;
            rc = trial(t, &ms);
            if (rc == ORBG_OK && ms < cur_ms) {
                cur = t;
                cur_ms = ms;
            }
        }
      }
      if (std::memcmp(&before, &cur, sizeof(cur)) == 0)
          break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != ORBG_OK)
        return rc;
    set->tuning = cur;
    if (best)
        *best = cur;
    /* leave the outputs holding the sample's results under the chosen tuning */
    return orbg_decode_batched(set, code_id, llr_offset, llr, B, query_cap, codeword, cw_offset,
                               queries, abandoned, cuda_stream);
}

}  // extern "C"

/* ------------------------------------------ per-block one-line fitting -- */

/*
 * Full ORBGRAND with one line fitted per block (Sec. III-E, then the order
 * of Sec. III-D).  With one line the fit gives beta = 1 and J_0 = [L_1/Q] -
 * 1 >= -1, so the blocks of a batch fall into few orders (one per J_0).
 * The object keeps one handle of the code per J_0 met so far, and a code
 * set over them; a decode fits every block on the device, marks which J_0s
 * occur (read back: one byte per possible J_0), adds the missing handles,
 * maps each block to its J_0's code id on the device, and decodes all
 * blocks in one batched launch.  J_0 above n(n+1)/2 orders patterns by Hamming weight
 * first whatever its value, so it is held at n(n+1)/2 + 1.
 */
struct orbg_fitted {
    const orbg_code *code;         /* not owned */
    int divisible;
    std::mutex mu;
    std::map<int32_t, int> slot;   /* J_0 -> index into handles */
    std::vector<orbg_code *> handles;
    orbg_codeset *set = nullptr;   /* over handles; rebuilt when one is added */
};

namespace {

/* The code in the one-line order of (J_0, beta = 1): line tables when
 * 0 <= J_0 <= ORBG_MAX_LINE and they reach the cap (a large J_0 takes them
 * past logistic weight ORBG_MAX_LOGISTIC), else the one-segment model
 * tables, which hold any weight. */
int fitted_handle(const orbg_code *code, int32_t J0, orbg_code **out)
{
    if (J0 >= 0 && J0 <= ORBG_MAX_LINE) {
        const int rc = load_code(code->H.data(), ORBG_MAT_H, code->n, code->k, code->max_cap,
                                 nullptr, J0, 1, out);
        if (rc != ORBG_ELIMIT)
            return rc;
    }
    OrbgModel md;
    md.m = 1;
    md.I[0] = 0;
    md.I[1] = code->n;
    md.J[0] = J0;
    md.beta[0] = 1;
    return load_code(code->H.data(), ORBG_MAT_H, code->n, code->k, code->max_cap, &md, 0, 1,
                     out);
}

}  // namespace

extern "C" {

int orbg_fitted_create(const orbg_code *code, int divisible, orbg_fitted **out)
{
    if (!out)
        return ORBG_EINVAL;
    *out = nullptr;
    if (!code)
        return ORBG_EINVAL;
    orbg_fitted *f = new (std::nothrow) orbg_fitted();
    if (!f)
        return ORBG_ENOMEM;
    f->code = code;
    f->divisible = divisible ? 1 : 0;
    *out = f;
    return ORBG_OK;
}

int orbg_fitted_free(orbg_fitted *f)
{
    if (!f)
        return ORBG_OK;
    orbg_codeset_free(f->set);
    for (orbg_code *c : f->handles)
        orbg_free_code(c);
    delete f;
    return ORBG_OK;
}

int orbg_fitted_decode(orbg_fitted *f, const float *llr, int64_t B, uint32_t query_cap,
                       uint8_t *codeword, uint32_t *queries, uint8_t *abandoned,
                       int32_t *models, void *cuda_stream)
{
    OrbgRange range("orbg_fitted_decode");
    if (!f || B < 0 || query_cap < 1)
        return ORBG_EINVAL;
    if (query_cap > f->code->max_cap || B >= ((int64_t)1 << 32))
        return ORBG_ELIMIT;
    if (B == 0)
        return ORBG_OK;
    if (!llr || !codeword || !queries || !abandoned || !is_device_ptr(llr) ||
        !is_device_ptr(codeword) || !is_device_ptr(queries) || !is_device_ptr(abandoned) ||
        !is_device_ptr(models))
        return ORBG_EINVAL;
    std::lock_guard<std::mutex> lk(f->mu);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int n = f->code->n;
    const int32_t top = n * (n + 1) / 2 + 1; /* J_0 held at most here */
    const size_t nj = (size_t)top + 2;       /* J_0 = -1 .. top */
    int32_t *d_models = models;
    int32_t *d_cid = nullptr, *d_lut = nullptr;
    uint8_t *d_present = nullptr;
    cudaError_t e = cudaSuccess;
    int rc = ORBG_OK;
    if ((!models && (e = alloc_async(&d_models,
                                         (size_t)B * ORBG_FIT_STRIDE * sizeof(int32_t), st)) !=
                        cudaSuccess) ||
        (e = alloc_async(&d_cid, (size_t)B * sizeof(int32_t), st)) != cudaSuccess ||
        (e = alloc_async(&d_lut, nj * sizeof(int32_t), st)) != cudaSuccess ||
        (e = alloc_async(&d_present, nj, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_present, 0, nj, st)) != cudaSuccess)
        rc = cuda_fail(e);
    /* every block's line, then which J_0s occur (device), read back */
    std::vector<uint8_t> present(nj);
    if (rc == ORBG_OK &&
        ((e = (cudaError_t)orbg_fit_launch(llr, B, n, 1, f->divisible, d_models,
                                           cuda_stream)) != cudaSuccess ||
         (e = (cudaError_t)orbg_fit_mark_lines(d_models, B, top, d_present, cuda_stream)) !=
             cudaSuccess ||
         (e = cudaMemcpyAsync(present.data(), d_present, nj, cudaMemcpyDeviceToHost, st)) !=
             cudaSuccess ||
         (e = cudaStreamSynchronize(st)) != cudaSuccess))
        rc = cuda_fail(e);
    /* a handle per J_0 met (cached across calls), and the J_0 -> code id table */
    std::vector<int32_t> lut(nj, 0);
    bool grown = false;
    for (size_t i = 0; i < nj && rc == ORBG_OK; i++) {
        if (!present[i])
            continue;
        const int32_t J0 = (int32_t)i - 1;
        auto it = f->slot.find(J0);
        if (it == f->slot.end()) {
            if (f->handles.size() >= 1024) {
                rc = ORBG_ELIMIT;
                break;
            }
            orbg_code *h = nullptr;
            if ((rc = fitted_handle(f->code, J0, &h)) != ORBG_OK)
                break;
            f->handles.push_back(h);
            it = f->slot.emplace(J0, (int)f->handles.size() - 1).first;
            grown = true;
        }
        lut[i] = it->second;
    }
    if (grown || !f->set) {
        /* a handle added in this call (even one that then failed on a
         * later J_0) makes the set stale: drop it, so that no call decodes
         * with a set that lacks a handle the J_0 map already names */
        orbg_codeset_free(f->set);
        f->set = nullptr;
        if (rc == ORBG_OK)
            rc = orbg_codeset_create(f->handles.data(), (int)f->handles.size(), &f->set);
    }
    /* code ids on the device, then one batched launch, each block in its
     * own line's order */
    if (rc == ORBG_OK &&
        ((e = cudaMemcpyAsync(d_lut, lut.data(), nj * sizeof(int32_t), cudaMemcpyHostToDevice,
                              st)) != cudaSuccess ||
         (e = (cudaError_t)orbg_fit_map_lines(d_models, B, top, d_lut, d_cid, cuda_stream)) !=
             cudaSuccess))
        rc = cuda_fail(e);
    /* the batched launch on device buffers (dense layout: every handle has
     * the code's n), as orbg_decode_batched makes it */
    unsigned long long *scratch = nullptr;
    if (rc == ORBG_OK &&
        (e = alloc_async(&scratch, orbg_batched_scratch_bytes(B, f->set->ncodes), st)) !=
            cudaSuccess)
        rc = cuda_fail(e);
    if (rc == ORBG_OK) {
        const orbg_codeset *set = f->set;
        const orbg_tuning &t = set->tuning;
        OrbgBatchedArgs a{};
        a.d_codes = set->d_codes;
        a.code0 = &set->code0;
        a.ncodes = set->ncodes;
        a.n_max = set->n_max;
        a.w32_max = set->w32_max;
        a.var = set->var;
        a.has_stride = set->has_stride;
        a.code_id = d_cid;
        a.llr_off = nullptr;
        a.llr = llr;
        a.B = B;
        a.cap = query_cap;
        a.budget = t.warp_budget < query_cap ? t.warp_budget : query_cap;
        a.cw = codeword;
        a.cw_off = nullptr;
        a.q = queries;
        a.ab = abandoned;
        a.scratch = scratch;
        a.warps_per_cta = t.warps_per_cta;
        a.ctas_per_sm = t.ctas_per_sm;
        a.grab = t.blocks_per_grab;
        a.heavy_warps = t.heavy_warps;
        a.ntrip_max = set->ntrip_max;
        a.x3w_max = set->x3w_max;
        a.stream = st;
        const int le = orbg_launch_batched(a);
        if (le != 0)
            rc = cuda_fail((cudaError_t)le);
    }
    for (void *p : {(void *)scratch, (void *)d_cid, (void *)d_lut, (void *)d_present})
        if (p)
            cudaFreeAsync(p, st);
    if (!models && d_models)
        cudaFreeAsync(d_models, st);
    return rc;
}

}  // extern "C"

/* ------------------------------------- per-block fitted models, any lines -- */

extern "C" {

int orbg_decode_fitted(const orbg_code *code, const float *llr, int64_t B, uint32_t query_cap,
                       int lines, int divisible, uint8_t *codeword, uint32_t *queries,
                       uint8_t *abandoned, int32_t *models, void *cuda_stream)
{
    OrbgRange range("orbg_decode_fitted");
    if (!code || B < 0 || query_cap < 1 || lines < 1 || lines > ORBG_MAX_SEG)
        return ORBG_EINVAL;
    if (query_cap > ORBG_MAX_QUERY_CAP || B >= ((int64_t)1 << 40))
        return ORBG_ELIMIT;
    if (B == 0)
        return ORBG_OK;
    if (!llr || !codeword || !queries || !abandoned)
        return ORBG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t nb = (size_t)B * code->n;
    Stager sg(st);
    const float *d_llr;
    uint8_t *d_cw, *d_ab;
    uint32_t *d_q;
    int32_t *d_rec = nullptr;
    int rc;
    if ((rc = sg.add(llr, nb * sizeof(float), true, false, &d_llr)) ||
        (rc = sg.add(codeword, nb, false, true, &d_cw)) ||
        (rc = sg.add(queries, (size_t)B * sizeof(uint32_t), false, true, &d_q)) ||
        (rc = sg.add(abandoned, (size_t)B, false, true, &d_ab)) ||
        (rc = sg.add(models, models ? (size_t)B * ORBG_FIT_STRIDE * sizeof(int32_t) : 0, false,
                     true, &d_rec))) {
        sg.finish(false);
        return rc;
    }
    unsigned char *queue = nullptr; /* the decoder's scratch */
    cudaError_t e = alloc_async(&queue, orbg_fitsearch_scratch_bytes(B), st);
    if (e != cudaSuccess) {
        sg.finish(false);
        return cuda_fail(e);
    }
    const int n = code->n;
    const int div = divisible ? 1 : 0;
    int le;
    if (n <= 32)
        le = orbg_launch_fitsearch_k1(code->dev, d_llr, B, query_cap, lines, div, d_cw, d_q,
                                      d_ab, d_rec, queue, st);
    else if (n <= 64)
        le = orbg_launch_fitsearch_k2(code->dev, d_llr, B, query_cap, lines, div, d_cw, d_q,
                                      d_ab, d_rec, queue, st);
    else if (n <= 128)
        le = orbg_launch_fitsearch_k4(code->dev, d_llr, B, query_cap, lines, div, d_cw, d_q,
                                      d_ab, d_rec, queue, st);
    else
        le = orbg_launch_fitsearch_k8(code->dev, d_llr, B, query_cap, lines, div, d_cw, d_q,
                                      d_ab, d_rec, queue, st);
    cudaFreeAsync(queue, st);
    if (le != 0) {
        sg.finish(false);
        return cuda_fail((cudaError_t)le);
    }
    if (!sg.any())
        return ORBG_OK;
    rc = sg.finish(true);
    if (rc)
        return rc;
    if (!is_device_ptr(abandoned) && std::memchr(abandoned, ORBG_BLOCK_NAN, (size_t)B))
        return ORBG_ENAN;
    return ORBG_OK;
}

}  // extern "C"
