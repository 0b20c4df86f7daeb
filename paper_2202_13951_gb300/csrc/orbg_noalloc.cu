/*
 * orbg_noalloc.cu -- a batched decode entry point that allocates nothing.
 *
 * Some callers cannot allocate device memory once they are running: a
 * receiver that reserves all of its GPU memory at start-up and treats any
 * later allocation as a fault, or code that must not risk an allocation
 * blocking behind other work on the device while it holds a latency budget.
 * orbg_decode_batched allocates its scratch (queue counters and the list of
 * blocks left open by phase 1) on the stream for every call, so it is not
 * usable there.  orbg_decode_batched_noalloc runs the same two launches with
 * that scratch in a fixed array compiled into this library instead.
 *
 * The array is a file-scope __device__ variable: every GPU that loads the
 * library holds it (the batched form's scratch for ORBG_NOALLOC_MAX_BLOCKS
 * blocks of a set of up to 1024 codes: 12 bytes per block, 8,264 bytes of
 * counters and 8.5 MiB of handover records, 14.5 MiB + 16,480 B in all) until
 * the process exits.  Host code cannot use the variable's name as a
 * device address, so the first call on each device, with that device
 * current, asks the runtime for the address (cudaGetSymbolAddress) and keeps
 * it; later calls on that device reuse it.  The kept address belongs to the
 * device's primary context (the one the runtime API uses): it is not valid
 * after cudaDeviceReset, nor in a context the caller made with the driver
 * API on the same device, and this entry point must not be used there.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/orbg.h"
#include "orbg_internal.h"

namespace {

constexpr int kMaxDevices = 64;

/* Scratch shared by every no-alloc call on a device, laid out as
 * orbg_scratch_layout places it: counters, per-code counts and cursors, the
 * open-block list and phase 1's block order. */
constexpr size_t kScratchWords =
    (8 * ORBG_BATCHED_COUNTERS + 16 * (ORBG_MAX_CODES + 1) + 12 * (size_t)ORBG_NOALLOC_MAX_BLOCKS +
     15 + (size_t)ORBG_HANDOVER_BYTES * ORBG_HANDOVER_MAX + 7) / 8;
static __device__ __align__(256) unsigned long long g_orbg_noalloc_scratch[kScratchWords];

std::mutex g_mu;
unsigned long long *g_scratch_addr[kMaxDevices];

/* Device address of the scratch array on the current device, looked up once
 * per device. Returns a cudaError_t value. */
int scratch_on_current_device(unsigned long long **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return (int)e;
    if (dev < 0 || dev >= kMaxDevices)
        return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_orbg_noalloc_scratch);
        if (e != cudaSuccess)
            return (int)e;
        g_scratch_addr[dev] = (unsigned long long *)p;
    }
    *out = g_scratch_addr[dev];
    return 0;
}

bool on_device(const void *p)
{
    if (!p)
        return true;
    /* clear only the probe's own error, never one the caller left pending */
    const cudaError_t pending = cudaPeekAtLastError();
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        if (pending == cudaSuccess)
            cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int orbg_decode_batched_noalloc(const orbg_codeset *set, const int32_t *code_id,
                                           const int64_t *llr_offset, const float *llr,
                                           int64_t B, uint32_t query_cap, uint8_t *codeword,
                                           const int64_t *cw_offset, uint32_t *queries,
                                           uint8_t *abandoned, void *cuda_stream)
{
    OrbgSetView v;
    if (!set || B < 0 || query_cap < 1 || orbg_codeset_view(set, &v) != 0)
        return ORBG_EINVAL;
    if (B > ORBG_NOALLOC_MAX_BLOCKS || query_cap > v.cap_min)
        return ORBG_ELIMIT;
    if (B == 0)
        return ORBG_OK;
    if (!llr || !codeword || !queries || !abandoned ||
        (llr_offset == nullptr) != (cw_offset == nullptr))
        return ORBG_EINVAL;
    /* staging host buffers would need an allocation: device buffers only */
    if (!on_device(llr) || !on_device(codeword) || !on_device(queries) ||
        !on_device(abandoned) || !on_device(code_id) || !on_device(llr_offset) ||
        !on_device(cw_offset))
        return ORBG_EINVAL;
    unsigned long long *scratch = nullptr;
    int e = scratch_on_current_device(&scratch);
    if (e != 0)
        return orbg_note_cuda_error(e);
    const uint32_t budget = v.tuning.warp_budget < query_cap ? v.tuning.warp_budget : query_cap;
    /* the launcher zeroes the counters on the stream before phase 1 */
    OrbgBatchedArgs a{};
    a.d_codes = v.d_codes;
    a.code0 = &v.code0;
    a.ncodes = v.ncodes;
    a.n_max = v.n_max;
    a.var = v.var;
    a.has_stride = v.has_stride;
    a.w32_max = v.w32_max;
    a.code_id = code_id;
    a.llr_off = llr_offset;
    a.llr = llr;
    a.B = B;
    a.cap = query_cap;
    a.budget = budget;
    a.cw = codeword;
    a.cw_off = cw_offset;
    a.q = queries;
    a.ab = abandoned;
    a.scratch = scratch;
    a.warps_per_cta = v.tuning.warps_per_cta;
    a.ctas_per_sm = v.tuning.ctas_per_sm;
    a.grab = v.tuning.blocks_per_grab;
    a.heavy_warps = v.tuning.heavy_warps;
    a.ntrip_max = v.ntrip_max;
    a.x3w_max = v.x3w_max;
    a.stream = cuda_stream;
    e = orbg_launch_batched(a);
    return e != 0 ? orbg_note_cuda_error(e) : ORBG_OK;
}
