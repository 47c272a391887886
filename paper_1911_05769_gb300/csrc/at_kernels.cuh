// at_kernels.cuh -- persistent weakly-synchronous AT stepper for sm_103a.
//
// One cooperative launch advances the whole 1D field by n_steps forward-Euler
// steps (arXiv 1911.05769, Sec. 3.2).  CTA c owns the contiguous subdomains
// [lo, hi) and sweeps them in step-major order.  A "tile" is one subdomain j
// over one pass of `len` consecutive levels n .. n+len (len = 1 except in
// blocked free-running mode).  Each CTA runs
//   * one producer warp: for tile r it copies the subdomain's M state words
//     and the neighbours' delayed boundary values (levels n-k-m, Eq. AT1/AT2)
//     from the ring buffers into shared-memory stage r % PD with cp.async,
//     after choosing the delays k (prescribed, replayed, or -- free running --
//     read off the neighbour's progress flag, waiting only while the neighbour
//     lags by more than the delay bound allows: the blocking branch of
//     Algorithm 2);
//   * four consumer warps: the halo approximation ("approximate" step of
//     Algorithm 2, split form of Sec. 5.2), the unchanged central stencil of
//     order 2 or 4 and the Euler update, `len` times on the tile held in
//     shared memory, the final level written back in place; after every level
//     the new boundary values go into ring slot (level mod T), followed, on
//     the CTA's two edge faces, by a release store of the progress flag (the
//     notified put).
// Halo values never come from the neighbour's state array, only from the
// ring, so each CTA updates its own subdomains in place.  Stage reuse is
// signalled with mbarriers (full: copies landed; empty: tile consumed).
//
// Blocked free-running mode (temporal blocking): a pass of len <= L+1 levels
// uses, at inner step i, the halo extrapolated with delay k0 + i from the
// levels available when the pass started (Eq. AT1/AT2 with a larger k), so
// the state is read and written once per pass instead of once per level.
//
// AT_SYNC replaces the flag waits with a grid barrier between steps
// (Algorithm 1).  Every wait is bounded by timeout_ns; on expiry the kernel
// latches AT_ERR_TIMEOUT in the control block, raises the abort word and
// every CTA leaves its loops.  Abort is uniform inside a CTA: the producer
// lets all its copies land before it raises the CTA's abort word, so every
// consumer sees the same set of completed stages and takes the same named
// barriers.
#pragma once

#include "at_device.cuh"

namespace atk {

constexpr int kConsumerWarps = 4;
constexpr int kConsumers = 32 * kConsumerWarps;   // threads 0..127
constexpr int kThreads = kConsumers + 32;         // + one producer warp
constexpr int kRingEntry = 16;                    // bytes per (slot, subdomain, face)
constexpr int kMaxS = 3;                          // levels per halo approximation
// stage layout: [0,16) header (k0 face 0, k0 face 1, len) | [16,112) delayed
// ring levels [face][m] | [112,128) left halo pad | tile (M words) | 16-byte
// right halo pad
constexpr int kRawOff = 16;
constexpr int kTileOff = 128;
constexpr int kPadBytes = 16;
constexpr int kMaxL = 16;
constexpr int kFullArrivals = 32 + 2;             // 32 copy arrivals + 2 header writers
constexpr int kMiscBytes = 256;                   // abort word + delay histograms
constexpr int kConsumerBarrier = 1;               // named barrier id of the consumer warps

enum : int { kModeSync = 0, kModeSeeded = 1, kModeFree = 2, kModeReplay = 3 };
enum : int {
    kCtrlStatus = 0, kCtrlAbort = 1, kCtrlCta = 2, kCtrlWhere = 3, kCtrlNb = 4, kCtrlStep = 5,
    kCtrlWords = 16
};
enum : int { kWhereFull = 1, kWhereEmpty = 2, kWhereFlag = 3, kWhereGrid = 4 };
constexpr int kStatusTimeout = -5;

// Shared-memory layout of the stepper, shared by the host (launch set-up) and
// the kernel.
struct SmemLayout {
    long long stage_bytes, stage_off, work_off, tab_off, total;
};

__host__ __device__ inline long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(long long M, int word, int stages, bool work, long long tab_words)
{
    SmemLayout l;
    l.stage_bytes = round_up(kTileOff + M * word + kPadBytes, 128);
    l.stage_off = round_up(16LL * stages + kMiscBytes, 128);
    l.work_off = l.stage_off + (long long)stages * l.stage_bytes;
    l.tab_off = l.work_off + (work ? l.stage_bytes : 0);
    l.total = l.tab_off + tab_words * word;
    return l;
}

struct Params {
    void *u;                   // state, N words, updated in place
    unsigned char *ring;       // [T][P][2] entries of 16 bytes
    unsigned long long *flag;  // [P][2] last level published per face
    int *ctrl;                 // control block (status, abort, diagnostics)
    unsigned long long *hist;  // [L+1] delay counts
    unsigned long long *gbar;  // grid-barrier arrival counter (AT_SYNC)
    int8_t *delays;            // [n_steps][P][2] replay input / record output
    long long N, P, M;
    int L, T, mode, per_sub;
    long long n0, n_steps;
    int sb;                    // levels per pass (temporal blocking, free mode)
    unsigned long long seed;
    double cA, cB, dtA;        // dt/(2dx) | dt/(12dx);  nu dt/dx^2 | nu dt/(12dx^2);  dt A
    double x0, dx;
    int forcing;
    int G;                     // CTAs
    int stages;                // stage buffers per CTA
    long long stage_bytes, stage_off, work_off, tab_off;
    long long timeout_ns;
    unsigned long long gbar_base;
    int skip_publish;          // test knob: CTA 0 stops releasing flags
    long long skip_step;
};

// ---------------------------------------------------------------------------
// bounded waits
// ---------------------------------------------------------------------------
__device__ __noinline__ void raise_timeout(const Params &p, int where, long long n, long long nb)
{
    if (atomicCAS(p.ctrl + kCtrlStatus, 0, kStatusTimeout) == 0) {
        p.ctrl[kCtrlCta] = (int)blockIdx.x;
        p.ctrl[kCtrlWhere] = where;
        p.ctrl[kCtrlNb] = (int)nb;
        p.ctrl[kCtrlStep] = (int)n;
    }
    atomicExch(p.ctrl + kCtrlAbort, 1);
}

// Producer side: waits for a stage to be released by the consumers.
__device__ __forceinline__ bool wait_mbar(uint64_t *bar, unsigned parity, const Params &p,
                                          volatile int *s_abort, int where, long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*s_abort) return false;
        if ((long long)(global_ns() - t0) > limit_ns) {
            raise_timeout(p, where, -1, -1);
            return false;
        }
    }
}

// Consumer side: waits for a stage to be filled.  Gives up only when the
// producer has raised the CTA's abort word, after re-testing the phase: the
// producer raises it only once all its copies have landed, so all consumers
// see the same completed phases and leave at the same tile.  The time limit
// is a last resort far beyond any producer wait.
__device__ __forceinline__ bool wait_full(uint64_t *bar, unsigned parity, const Params &p,
                                          volatile int *s_abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*s_abort) {
            __threadfence_block();
            return mbar_try_wait(bar, parity);
        }
        if ((long long)(global_ns() - t0) > 16 * p.timeout_ns) {
            raise_timeout(p, kWhereFull, -1, -1);
            return false;
        }
    }
}

// Waits until *fl >= need (acquire).  Returns the value seen in *seen.
__device__ __noinline__ bool wait_flag(const Params &p, const unsigned long long *fl, long long need,
                                       unsigned long long *seen, long long n, long long nb)
{
    unsigned long long v = ld_acquire(fl);
    if ((long long)v >= need) { *seen = v; return true; }
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        v = ld_acquire(fl);
        if ((long long)v >= need) { *seen = v; return true; }
        if (ld_relaxed(p.ctrl + kCtrlAbort)) return false;
        if ((long long)(global_ns() - t0) > p.timeout_ns) {
            raise_timeout(p, kWhereFlag, n, nb);
            return false;
        }
    }
}

__device__ __noinline__ bool wait_grid(const Params &p, unsigned long long target, long long n)
{
    if (ld_acquire(p.gbar) >= target) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        __nanosleep(20);
        if (ld_acquire(p.gbar) >= target) return true;
        if (ld_relaxed(p.ctrl + kCtrlAbort)) return false;
        if ((long long)(global_ns() - t0) > p.timeout_ns) {
            raise_timeout(p, kWhereGrid, n, -1);
            return false;
        }
    }
}

__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync %0, %1;" ::"n"(kConsumerBarrier), "n"(kConsumers) : "memory");
}

// ---------------------------------------------------------------------------
// shared-memory vector access
// ---------------------------------------------------------------------------
template <typename T, int CNT>
__device__ __forceinline__ void lds(const T *s, T *v)
{
    if constexpr (sizeof(T) == 4 && CNT == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(s);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if constexpr (sizeof(T) == 4 && CNT == 2) {
        const float2 a = *reinterpret_cast<const float2 *>(s);
        v[0] = a.x; v[1] = a.y;
    } else if constexpr (sizeof(T) == 8 && CNT == 4) {
        const double2 a = *reinterpret_cast<const double2 *>(s);
        const double2 b = *reinterpret_cast<const double2 *>(s + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else if constexpr (sizeof(T) == 8 && CNT == 2) {
        const double2 a = *reinterpret_cast<const double2 *>(s);
        v[0] = a.x; v[1] = a.y;
    } else {
#pragma unroll
        for (int i = 0; i < CNT; ++i) v[i] = s[i];
    }
}

template <typename T>
__device__ __forceinline__ void sts4(T *s, const T *v)
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(s) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *reinterpret_cast<double2 *>(s) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(s + 2) = make_double2(v[2], v[3]);
    }
}

// 4 consecutive words to global memory (16-byte aligned), bypassing L1.
template <typename T>
__device__ __forceinline__ void stg4(T *g, const T *v)
{
    if constexpr (sizeof(T) == 4) {
        st_cg16(g, v[0], v[1], v[2], v[3]);
    } else {
        st_cg16(g, v[0], v[1]);
        st_cg16(g + 2, v[2], v[3]);
    }
}

// One 16-byte ring entry holding R words (the rest zero).
template <typename T, int R>
__device__ __forceinline__ void st_entry(unsigned char *e, const T *v)
{
    if constexpr (sizeof(T) == 4) {
        st_cg16(e, v[0], R > 1 ? v[1] : 0.0f, 0.0f, 0.0f);
    } else {
        st_cg16(e, v[0], R > 1 ? v[1] : 0.0);
    }
}

// Halo approximation from s delayed levels raw[m] = f^{n-k-m} (16-byte
// entries, word r of each): Lagrange extrapolation in time to level n.
// s = 2 gives (k+1) f^{n-k} - k f^{n-k-1} (Eq. AT1/AT2); s = 3 uses the
// quadratic through n-k, n-k-1, n-k-2.  k = 0 returns f^n itself.
template <typename T, int S_LEV>
__device__ __forceinline__ T approx_halo(const unsigned char *raw, int k, int r)
{
    const T r0 = reinterpret_cast<const T *>(raw)[r];
    if (k == 0) return r0;
    const T r1 = reinterpret_cast<const T *>(raw + kRingEntry)[r];
    if constexpr (S_LEV == 2) {
        return (T)(k + 1) * r0 - (T)k * r1;
    } else {
        const T r2 = reinterpret_cast<const T *>(raw + 2 * kRingEntry)[r];
        const T w0 = (T)((k + 1) * (k + 2) / 2);
        const T w1 = (T)(-k * (k + 2));
        const T w2 = (T)(k * (k + 1) / 2);
        return w0 * r0 + w1 * r1 + w2 * r2;
    }
}

// ---------------------------------------------------------------------------
// producer warp
// ---------------------------------------------------------------------------
template <typename T, int ORDER>
__device__ void produce(const Params &p, long long lo, long long hi, int PD, uint64_t *full, uint64_t *empty,
                        volatile int *s_abort, unsigned char *stages, unsigned *s_hist)
{
    constexpr int S_LEV = ORDER / 2 + 1;
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long S = hi - lo;
    const long long n_end = p.n0 + p.n_steps;
    const int chunks = (int)(p.M * (long long)sizeof(T) / 16);
    const size_t tile_bytes = (size_t)p.M * sizeof(T);
    const size_t slot_stride = (size_t)p.P * 2 * kRingEntry;
    unsigned *my_hist = s_hist + (lane & 1) * (kMaxL + 1);   // lanes 0 and 1 only

    int kb = 0;                 // lane i: raw delay of (tile r0 + i/2, face i%2) of the batch
    int st = 0;                 // stage of tile r
    unsigned use = 0;           // r / PD
    long long n = p.n0, j = lo; // pass start level and subdomain of tile r
    long long r = 0;
    bool ok = true;

    while (n < n_end) {
        // levels in this pass: passes longer than one level extrapolate from s
        // levels, so they start only once level s-1 exists (the same rule in
        // every CTA, so all agree on the pass boundaries)
        int len = (int)((n_end - n) < p.sb ? (n_end - n) : p.sb);
        if (n < S_LEV - 1) len = 1;
        // every 16 tiles, the 32 lanes draw the 32 (tile, face) delays at
        // once (prescribed modes, one level per pass)
        if ((r & 15) == 0 && (p.mode == kModeSeeded || p.mode == kModeReplay)) {
            long long jj = j + (lane >> 1), nn = n;
            while (jj >= hi) { jj -= S; ++nn; }
            const int f = lane & 1;
            int k = 0;
            if (nn < n_end) {
                if (p.mode == kModeSeeded)
                    k = seeded_delay(p.seed, nn, jj, p.P, p.per_sub ? 0 : f, p.L);
                else
                    k = p.delays[((nn - p.n0) * p.P + jj) * 2 + f];
            }
            kb = k;
        }
        if (r >= PD) {
            // lane 0 waits for the consumers to release the stage, then the
            // whole warp may overwrite it
            int freed = 1;
            if (lane == 0) freed = wait_mbar(&empty[st], (use - 1u) & 1u, p, s_abort, kWhereEmpty, 8 * p.timeout_ns);
            freed = __shfl_sync(kAll, freed, 0);
            __syncwarp();
            if (!freed) { ok = false; break; }
        }
        const long long step = n - p.n0;
        unsigned char *sb = stages + (size_t)st * p.stage_bytes;

        // synchronous algorithm: every halo of step n waits for all CTAs to
        // have finished step n-1 (grid barrier, Algorithm 1)
        if (p.mode == kModeSync && step > 0 && j == lo) {
            int good = 1;
            if (lane == 0)
                good = wait_grid(p, p.gbar_base + (unsigned long long)step * (unsigned long long)p.G, n);
            good = __shfl_sync(kAll, good, 0);
            if (!good) { ok = false; break; }
        }

        // state tile of subdomain j at level n
        const unsigned char *src = reinterpret_cast<const unsigned char *>(p.u) + (size_t)j * tile_bytes;
        for (int q = lane; q < chunks; q += 32) cp_async16(sb + kTileOff + 16 * q, src + 16 * q);

        // delays and delayed ring levels, lane f for face f
        const int bi = 2 * (int)(r & 15);
        const int kr0 = __shfl_sync(kAll, kb, bi);
        const int kr1 = __shfl_sync(kAll, kb, bi + 1);
        int good = 1;
        if (lane < 2) {
            const int f = lane;
            const long long q = (f == 0) ? (j == 0 ? p.P - 1 : j - 1) : (j == p.P - 1 ? 0 : j + 1);
            // The CTA's two edge faces always use the progress flags, also when
            // the neighbour is the same CTA (one CTA, periodic wrap): there the
            // neighbour's level n comes from the tile just before this one.
            const bool cross = (f == 0) ? (j == lo) : (j == hi - 1);
            // largest delay at the start of the pass such that the last inner
            // step stays within L, and no level below 0 is ever read
            long long kmax = n - S_LEV + 1;
            if (kmax < 0) kmax = 0;
            if (kmax > p.L - (len - 1)) kmax = p.L - (len - 1);
            long long k = f ? kr1 : kr0;
            if (p.mode == kModeFree || p.mode == kModeSync) k = 0;
            if (k > kmax) k = kmax;
            if (k < 0) k = 0;
            if (cross && p.mode != kModeSync) {
                const unsigned long long *fl = p.flag + q * 2 + (1 - f);
                const long long need = (p.mode == kModeFree) ? n - kmax : n - k;
                unsigned long long seen = 0;
                if (!wait_flag(p, fl, need, &seen, n, q)) {
                    good = 0;
                } else if (p.mode == kModeFree) {
                    const long long avail = ((long long)seen < n) ? (long long)seen : n;
                    k = n - avail;
                }
            }
            if (good) {
                for (int i = 0; i < len; ++i) {
                    my_hist[k + i] += 1u;
                    if (p.delays && p.mode != kModeReplay)
                        p.delays[((step + i) * p.P + j) * 2 + f] = (int8_t)(k + i);
                }
                reinterpret_cast<volatile int *>(sb)[f] = (int)k;
                if (f == 0) reinterpret_cast<volatile int *>(sb)[2] = len;
                const unsigned char *rbase = p.ring + ((size_t)q * 2 + (1 - f)) * kRingEntry;
                const int levels = (k == 0 && len == 1) ? 1 : S_LEV;
                for (int m = 0; m < levels; ++m) {
                    const long long lv = n - k - m;
                    cp_async16(sb + kRawOff + (f * kMaxS + m) * kRingEntry,
                               rbase + (size_t)(lv & (p.T - 1)) * slot_stride);
                }
            }
        }
        good = __all_sync(kAll, good);
        if (!good) { ok = false; break; }
        mbar_arrive_on_copies(&full[st]);
        if (lane < 2) mbar_arrive(&full[st]);

        ++r;
        if (++st == PD) { st = 0; ++use; }
        if (++j == hi) { j = lo; n += len; }
    }
    // let every issued copy land, and the stage phases they complete become
    // visible, before the abort word is raised: consumers then agree on which
    // stages are complete and leave at the same tile
    cp_async_wait_all();
    __syncwarp();
    if (!ok) {
        if (lane == 0) {
            const long long first = r > PD ? r - PD : 0;
            for (long long q = first; q < r; ++q) {
                const unsigned long long t0 = global_ns();
                while (!mbar_try_wait(&full[q % PD], (unsigned)((q / PD) & 1)) &&
                       (long long)(global_ns() - t0) < p.timeout_ns) {
                }
            }
            __threadfence_block();
            *s_abort = 1;
        }
        __syncwarp();
    }
    if (lane < 2) {
        for (int i = 0; i <= p.L && i <= kMaxL; ++i)
            if (my_hist[i]) atomicAdd(p.hist + i, (unsigned long long)my_hist[i]);
    }
}

// ---------------------------------------------------------------------------
// consumer warps
// ---------------------------------------------------------------------------
template <typename T, int ORDER>
__device__ void consume(const Params &p, long long lo, long long hi, int PD, uint64_t *full, uint64_t *empty,
                        volatile int *s_abort, unsigned char *stages, unsigned char *work, const T *tab)
{
    constexpr int R = ORDER / 2;
    constexpr int S_LEV = ORDER / 2 + 1;
    constexpr int NV = 4 + 2 * R;
    const int t = threadIdx.x;
    const long long S = hi - lo;
    const long long n_end = p.n0 + p.n_steps;
    const int NG = (int)(p.M / 4);
    const T cA = (T)p.cA, cB = (T)p.cB, dtA = (T)p.dtA;
    const size_t slot_stride = (size_t)p.P * 2 * kRingEntry;
    const T *sj = tab, *cj = tab + p.M, *spt = tab + 2 * p.M, *cpt = spt + S;
    T *wtile = reinterpret_cast<T *>(work + kTileOff);

    int st = 0;
    unsigned use = 0;
    long long n = p.n0, j = lo;
    while (n < n_end) {
        if (!wait_full(&full[st], use & 1u, p, s_abort)) break;
        const unsigned char *sb = stages + (size_t)st * p.stage_bytes;
        T *stile = reinterpret_cast<T *>(const_cast<unsigned char *>(sb) + kTileOff);
        const int k0 = reinterpret_cast<const volatile int *>(sb)[0];
        const int k1 = reinterpret_cast<const volatile int *>(sb)[1];
        const int len = reinterpret_cast<const volatile int *>(sb)[2];
        T sp = 0, cp = 0;
        if (p.forcing) { sp = spt[j - lo]; cp = cpt[j - lo]; }
        T *ug = reinterpret_cast<T *>(p.u) + (size_t)j * p.M;
        const bool edge_pub = !(p.skip_publish && blockIdx.x == 0);

        for (int i = 0; i < len; ++i) {
            const T *src = (i & 1) ? wtile : stile;
            T *dst = (i & 1) ? stile : wtile;
            const bool last = (i == len - 1);
            const long long lev = n + i + 1;                 // level being computed
            const long long slot = lev & (p.T - 1);
            const bool pub_ok = edge_pub || lev <= p.skip_step;
            for (int g = t; g < NG; g += kConsumers) {
                T v[NV];
                lds<T, 4>(src + 4 * g, v + R);
                if (g == 0 && i == 0) {
#pragma unroll
                    for (int q = 0; q < R; ++q) v[q] = approx_halo<T, S_LEV>(sb + kRawOff, k0, q);
                } else {
                    lds<T, R>(src + 4 * g - R, v);   // inner steps: halo sits in the pad
                }
                if (g == NG - 1 && i == 0) {
#pragma unroll
                    for (int q = 0; q < R; ++q)
                        v[R + 4 + q] = approx_halo<T, S_LEV>(sb + kRawOff + kMaxS * kRingEntry, k1, q);
                } else {
                    lds<T, R>(src + 4 * g + 4, v + R + 4);
                }
                T fo[4] = {0, 0, 0, 0};
                if (p.forcing) {
                    T s4[4], c4[4];
                    lds<T, 4>(sj + 4 * g, s4);
                    lds<T, 4>(cj + 4 * g, c4);
#pragma unroll
                    for (int e = 0; e < 4; ++e) fo[e] = dtA * (sp * c4[e] + cp * s4[e]);
                }
                T out[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const T c = v[e + R];
                    T a, b;
                    if constexpr (ORDER == 2) {
                        a = v[e + 2] - v[e];
                        b = (v[e + 2] + v[e]) - (T)2 * c;
                    } else {
                        a = (T)8 * (v[e + 3] - v[e + 1]) - (v[e + 4] - v[e]);
                        b = (T)16 * (v[e + 3] + v[e + 1]) - (v[e + 4] + v[e]) - (T)30 * c;
                    }
                    out[e] = c + ((cB * b - cA * c * a) + fo[e]);
                }
                if (last) stg4<T>(ug + 4 * g, out);
                else sts4<T>(dst + 4 * g, out);
                // publish the new boundary values and release the edge flag
                if (g == 0) {
                    unsigned char *e = p.ring + (size_t)slot * slot_stride + ((size_t)j * 2 + 0) * kRingEntry;
                    st_entry<T, R>(e, out);
                    if (p.mode == kModeSync) __threadfence();
                    if (j == lo && pub_ok) st_release(p.flag + j * 2 + 0, (unsigned long long)lev);
                    if (!last) {
                        // left halo of the next inner step, delay k0 + i + 1
#pragma unroll
                        for (int q = 0; q < R; ++q)
                            dst[q - R] = approx_halo<T, S_LEV>(sb + kRawOff, k0 + i + 1, q);
                    }
                }
                if (g == NG - 1) {
                    unsigned char *e = p.ring + (size_t)slot * slot_stride + ((size_t)j * 2 + 1) * kRingEntry;
                    st_entry<T, R>(e, out + 4 - R);
                    if (p.mode == kModeSync) __threadfence();
                    if (j == hi - 1 && pub_ok) st_release(p.flag + j * 2 + 1, (unsigned long long)lev);
                    if (!last) {
#pragma unroll
                        for (int q = 0; q < R; ++q)
                            dst[p.M + q] = approx_halo<T, S_LEV>(sb + kRawOff + kMaxS * kRingEntry, k1 + i + 1, q);
                    }
                }
            }
            if (!last) consumer_sync();
        }
        // synchronous algorithm: arrive at the grid barrier once the CTA has
        // finished step n (the consumers' named barrier orders their writes)
        if (p.mode == kModeSync && j == hi - 1) {
            consumer_sync();
            if (t == 0) {
                __threadfence();
                atomicAdd(p.gbar, 1ull);
            }
        }
        mbar_arrive(&empty[st]);
        if (++st == PD) { st = 0; ++use; }
        if (++j == hi) { j = lo; n += len; }
    }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <typename T, int ORDER>
__global__ void __launch_bounds__(kThreads, 2) at_stepper(const Params p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + p.stages;
    unsigned char *misc = reinterpret_cast<unsigned char *>(empty + p.stages);
    volatile int *s_abort = reinterpret_cast<volatile int *>(misc);
    unsigned *s_hist = reinterpret_cast<unsigned *>(misc + 16);     // [2][kMaxL+1]
    unsigned char *stages = smem + p.stage_off;
    unsigned char *work = smem + p.work_off;
    T *tab = reinterpret_cast<T *>(smem + p.tab_off);

    const long long c = blockIdx.x;
    const long long lo = c * p.P / p.G;
    const long long hi = (c + 1) * p.P / p.G;
    const long long S = hi - lo;
    // Stage r % PD may be refilled once tile r - PD is consumed; the refill
    // needs the state of tile r - S and the ring levels of tiles up to
    // r - S + 1, hence PD <= S - 1 (PD = 1 when S == 1).
    const int PD = (S <= 1) ? 1 : (int)((S - 1) < p.stages ? (S - 1) : p.stages);

    if (threadIdx.x == 0) {
        for (int i = 0; i < PD; ++i) {
            mbar_init(&full[i], kFullArrivals);
            mbar_init(&empty[i], kConsumers);
        }
        *s_abort = 0;
        mbar_fence_init();
    }
    if (threadIdx.x < 2 * (kMaxL + 1)) s_hist[threadIdx.x] = 0u;
    if (p.forcing) {
        // sin/cos of the offsets j dx within a subdomain and of the subdomain
        // origins x0 + p M dx (FP64), so that A sin(x_i) needs two FMAs
        for (long long i = threadIdx.x; i < p.M; i += blockDim.x) {
            double sv, cv;
            sincos((double)i * p.dx, &sv, &cv);
            tab[i] = (T)sv;
            tab[p.M + i] = (T)cv;
        }
        for (long long i = threadIdx.x; i < S; i += blockDim.x) {
            double sv, cv;
            sincos(p.x0 + (double)((lo + i) * p.M) * p.dx, &sv, &cv);
            tab[2 * p.M + i] = (T)sv;
            tab[2 * p.M + S + i] = (T)cv;
        }
    }
    __syncthreads();

    if (threadIdx.x >= kConsumers)
        produce<T, ORDER>(p, lo, hi, PD, full, empty, s_abort, stages, s_hist);
    else
        consume<T, ORDER>(p, lo, hi, PD, full, empty, s_abort, stages, work, tab);
}

// ---------------------------------------------------------------------------
// state (re)initialisation: level-0 boundary values into ring slot 0, flags 0
// ---------------------------------------------------------------------------
template <typename T, int R>
__global__ void at_init(const Params p)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < p.P; j += stride) {
        const T *u = reinterpret_cast<const T *>(p.u) + j * p.M;
        T a[2] = {u[0], R > 1 ? u[1] : (T)0};
        T b[2] = {u[p.M - R], R > 1 ? u[p.M - R + 1] : (T)0};
        st_entry<T, R>(p.ring + ((size_t)j * 2 + 0) * kRingEntry, a);
        st_entry<T, R>(p.ring + ((size_t)j * 2 + 1) * kRingEntry, b);
        p.flag[j * 2 + 0] = 0ull;
        p.flag[j * 2 + 1] = 0ull;
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x < kCtrlWords) p.ctrl[threadIdx.x] = 0;
        if (threadIdx.x <= p.L) p.hist[threadIdx.x] = 0ull;
        if (threadIdx.x == 0) *p.gbar = 0ull;
    }
}

}  // namespace atk
