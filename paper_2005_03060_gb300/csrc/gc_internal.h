// Internal declarations shared by the gridcorr CUDA translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gridcorr.h"

// device-side error bits (accumulated in gc_ctx::status_dev)
#define GC_DEV_TIMEOUT_FFT   0x1u
#define GC_DEV_TIMEOUT_XENG  0x2u
#define GC_DEV_TIMEOUT_CAL   0x4u
#define GC_DEV_BADINDEX      0x8u
#define GC_DEV_BADINPUT      0x10u   // zero or non-finite gain, non-finite sums

// bounded waits: give up after this many nanoseconds of %globaltimer
#define GC_WAIT_LIMIT_NS     1000000000ull

struct gc_prof_rec {
    const char *name;
    cudaEvent_t start, stop;
};

// tuning knobs (gc_set_tuning); 0 = automatic
enum {
    GC_TUNE_FFT_CHUNK = 0,
    GC_TUNE_XENG_TSPLIT = 1,
    GC_TUNE_CAL_CTAS = 2,
    GC_TUNE_CAL_ORDER = 3,
    GC_TUNE_CAL_OP = 4,
    GC_TUNE_XENG_PATH = 5,
    GC_TUNE_XENG_TC_SHAPE = 6,
    GC_TUNE_FFT_SHAPE = 7,
    GC_TUNE_FFT_PATH = 8,
    GC_TUNE_N = 9
};

// staging buffers of the streamed integration: with three, a chunk's copy
// may run two chunks ahead of the kernels
constexpr int GC_NSTAGE = 3;

struct gc_ctx {
    int device = 0;
    int tune[GC_TUNE_N] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int sm_count = 0;
    unsigned int *status_dev = nullptr;   // device error word
    void *scratch = nullptr;              // grow-only workspace
    size_t scratch_bytes = 0;
    std::string last_error;
    void *encode_tiled = nullptr;         // cuTensorMapEncodeTiled entry point
    // opt-in launch timing (gc_profile_enable): events around every launch
    bool profile = false;
    std::vector<gc_prof_rec> prof;        // records since the last read
    std::vector<cudaEvent_t> event_pool;
    // gc_integrate_host: copy stream, two device staging buffers, events
    cudaStream_t copy_stream = nullptr;
    void *stage[GC_NSTAGE] = {nullptr, nullptr, nullptr};   // gc_integrate_host staging buffers
    size_t stage_bytes = 0;
    cudaEvent_t ev_copied[GC_NSTAGE] = {nullptr, nullptr, nullptr}, ev_free[GC_NSTAGE] = {nullptr, nullptr, nullptr};
    // gc_integrate_host with host-resident gains: their device copy and the
    // events that order it against the kernels reading it
    void *gains_dev[2] = {nullptr, nullptr};   // host gains staged on the device, alternate calls
    size_t gains_bytes = 0;
    int gains_slot = 0;
    cudaEvent_t ev_gains_copied = nullptr, ev_gains_free[2] = {nullptr, nullptr};
};

// launch timing helpers: no-ops unless profiling is enabled
int gc_prof_begin(gc_ctx *ctx, cudaStream_t s, const char *name);
void gc_prof_end(gc_ctx *ctx, cudaStream_t s, int rec);

// error helpers (gc_runtime.cu)
gc_status gc_fail(gc_ctx *ctx, gc_status st, const std::string &msg);
gc_status gc_cuda_fail(gc_ctx *ctx, cudaError_t e, const char *what);
gc_status gc_scratch_reserve(gc_ctx *ctx, size_t bytes);
bool gc_aligned(const void *p, size_t a);

// FFT-correlator with the row stage on the tensor cores (gc_fftcorr_tc.cu)
bool gc_fft_tc_eligible(const gc_ctx *ctx, int vfmt, int L, const void *volt, bool masked);
gc_status gc_fft_tc_run(gc_ctx *ctx, const void *volt, int L, int C, int T, const float *gains, float **ppart,
                        int *n_chunks, cudaStream_t stream);

// tensor-map encode through the driver entry point (no libcuda link)
gc_status gc_encode_tiled(gc_ctx *ctx, CUtensorMap *map, CUtensorMapDataType dt, int rank,
                          void *base, const uint64_t *dims, const uint64_t *strides_bytes,
                          const uint32_t *box);

// ------------------------------------------------------------------ device helpers
#ifdef __CUDACC__

__device__ __forceinline__ uint64_t gc_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t gc_smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void gc_mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gc_smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void gc_fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void gc_fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void gc_mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(gc_smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bounded parity wait: true when the phase completed, false when the
// %globaltimer budget ran out (the caller reports and stops).
__device__ __forceinline__ bool gc_mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    const uint32_t a = gc_smem_addr(bar);
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 0u) {
            uint64_t now = gc_globaltimer();
            if (it == 0u) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
}

__device__ __forceinline__ void gc_mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(gc_smem_addr(bar)) : "memory");
}

// Bounded parity wait that also gives up when another role has raised
// `*abort`; true when the phase completed.
__device__ __forceinline__ bool gc_mbar_wait_abort(uint64_t *bar, uint32_t parity, volatile int *abort,
                                                   uint64_t limit_ns) {
    const uint32_t a = gc_smem_addr(bar);
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63u) == 0u) {
            if (*abort) return false;
            const uint64_t now = gc_globaltimer();
            if (it == 0u) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
}

// 4-D tiled TMA load into shared memory, completing on `bar`.
__device__ __forceinline__ void gc_tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                               int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(gc_smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(gc_smem_addr(bar))
        : "memory");
}

// 1-D bulk copy global -> shared (size and both addresses 16-byte aligned).
__device__ __forceinline__ void gc_bulk_load(void *dst, const void *src, uint32_t bytes,
                                             uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(gc_smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(gc_smem_addr(bar))
        : "memory");
}

#endif  // __CUDACC__
