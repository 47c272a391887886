// at_device.cuh -- device primitives of the persistent AT stepper (sm_103a).
//
// Inline PTX for the pieces the kernel needs: shared-memory mbarriers
// (pipeline full/empty signalling), cp.async 16-byte copies whose completion
// arrives on an mbarrier, gpu-scope release/acquire on the progress flags
// (the device counterpart of the notified put / notification test of
// Algorithm 2), the global nanosecond timer that bounds every wait, and the
// SplitMix64 generator for prescribed delays.
#pragma once

#include <cstdint>

namespace atk {

// Control block words (the solver's workspace).  kCtrlN0 (64-bit, words 8-9)
// is the time level of the state: every launch reads it at its start and the
// last CTA to finish advances it, so that a launch replayed from a captured
// graph continues where the previous one stopped.  kCtrlDone counts finished
// CTAs.  A bounded wait that expires latches kStatusTimeout with where it
// happened and raises the abort word that every other wait polls.
enum : int {
    kCtrlStatus = 0, kCtrlAbort = 1, kCtrlCta = 2, kCtrlWhere = 3, kCtrlNb = 4, kCtrlStep = 5,
    kCtrlN0 = 8, kCtrlDone = 10, kCtrlWords = 16
};
enum : int { kWhereTile = 1, kWhereRing = 2, kWhereFlag = 3, kWhereGrid = 4, kWhereAdjoint = 5 };
constexpr int kStatusTimeout = -5;

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// ---- mbarrier -------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible before first use by other threads
// and by the asynchronous copy units.
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Regular arrival (release semantics at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Arrival triggered when all cp.async copies issued so far by this thread
// have landed; counts as one of the barrier's expected arrivals.
__device__ __forceinline__ void mbar_arrive_on_copies(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One bounded probe of the phase with the given parity (acquire at CTA scope).
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// ---- cp.async -------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src_gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem)
                 : "memory");
}

// ---- bulk copy (TMA engine, async proxy) -----------------------------------
// Arrival that also announces `bytes` of asynchronous transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Contiguous global -> shared copy of `bytes` (multiple of 16, both ends
// 16-byte aligned) whose completion is counted on `bar`.
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Tiled tensor copy (TMA): the box of a 3D tensor map at element coordinates
// (x, y, z) into shared memory, completion counted on `bar`.  x times the
// element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tensor_load_3d(void *dst_smem, const void *tmap, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst_smem)), "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// The same for a 4D tensor map (element coordinates x, y, z, w).
__device__ __forceinline__ void tensor_load_4d(void *dst_smem, const void *tmap, int x, int y, int z, int w,
                                               uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(smem_addr(dst_smem)), "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
        : "memory");
}

// Orders this thread's earlier generic-proxy global accesses before later
// async-proxy accesses (a bulk copy re-reading data written with st.global).
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---- gpu-scope release / acquire ------------------------------------------
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// CTA-scope release/acquire on a 64-bit shared-memory word (per-warp progress)
__device__ __forceinline__ void st_release_cta_shared(volatile long long *p, long long v)
{
    asm volatile("st.release.cta.shared.b64 [%0], %1;" ::"r"(smem_addr((const void *)p)), "l"(v) : "memory");
}

__device__ __forceinline__ long long ld_acquire_cta_shared(const volatile long long *p)
{
    long long v;
    asm volatile("ld.acquire.cta.shared.b64 %0, [%1];" : "=l"(v) : "r"(smem_addr((const void *)p)) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- 16-byte global stores that bypass L1 ----------------------------------
__device__ __forceinline__ void st_cg16(void *p, float a, float b, float c, float d)
{
    asm volatile("st.global.cg.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}
__device__ __forceinline__ void st_cg16(void *p, double a, double b)
{
    asm volatile("st.global.cg.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(a), "d"(b) : "memory");
}

// ---- SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) --------------------------
// i-th output (0-based) of the sequence started from state `seed`: the state
// advances by the golden-ratio increment 0x9E3779B97F4A7C15 and is mixed by
// xor-shift-multiply with (30, 0xBF58476D1CE4E5B9), (27, 0x94D049BB133111EB), 31.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long i)
{
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Prescribed delay in {0..L} for counter (n*P + p)*2 + face: upper 32 bits of
// the generator output scaled to L+1 values by a multiply-shift.
__device__ __forceinline__ int seeded_delay(unsigned long long seed, long long n, long long p, long long P,
                                            int face, int L)
{
    const unsigned long long ctr =
        ((unsigned long long)n * (unsigned long long)P + (unsigned long long)p) * 2ull + (unsigned long long)face;
    const unsigned long long h = splitmix64(seed, ctr) >> 32;
    return (int)((h * (unsigned long long)(L + 1)) >> 32);
}

}  // namespace atk
