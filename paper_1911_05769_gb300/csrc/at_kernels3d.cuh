// at_kernels3d.cuh -- persistent AT stepper for the scalar 3D Burgers equation
//     u_t + u (u_x + u_y + u_z) = nu (u_xx + u_yy + u_zz)
// (the scalar form of Eq. BS in three dimensions) on a periodic box, order-2
// central differences, AT halos on the six faces of every subdomain
// (Eq. AT1/AT2 in split form, Sec. 3.2).
//
// The state keeps its natural layout (x fastest).  Subdomains of m0 x m1 x m2
// points are numbered (p2 P1 + p1) P0 + p0.  Each CTA is one processing
// element owning the subdomains [lo, hi) and sweeps them level by level.  A
// tile (one subdomain at one level) is swept plane by plane along z: every
// plane (an m0 x m1 box) is brought into one of `stages` shared-memory buffers
// by one TMA tensor copy (3D tensor map over the state; completion counted on
// the stage's mbarrier), several planes ahead; the last warp to finish with a
// stage (a shared counter per stage) refills it.  A thread owns up to TC
// groups of VW consecutive (x, y) columns; it keeps the values of its columns
// at planes z-1, z in registers, reads the plane z+1 and the y neighbours as
// VW-word vectors, and the two x neighbours beyond a group by warp shuffles
// (VW = 4) or as single words from shared memory (VW = 1).  The halo planes
// of a tile are staged once at its start, face by face, one warp per face.
// Neighbours across a subdomain face come from the ring of face planes:
// entry [slot][subdomain][face] holds the face's boundary values at level
// slot (faces 0/1: the x = 0 / x = m0-1 planes indexed [z][y]; 2/3: y planes
// [z][x]; 4/5: z planes [y][x]), extrapolated with the face's delay k from
// levels n-k, n-k-1.  After a tile every face's progress flag is released.
// The update is written in place; the next read of a plane is a bulk copy,
// so writers fence the async proxy before it is issued.
//
// Delays: one per (level, subdomain, face): seeded (counter (n P + p) 6 + f),
// replayed, free-running (read off the neighbour's flag, waiting only while
// it lags by more than L), or zero with a grid barrier per level (Algorithm 1).
// Every wait is bounded; on expiry the kernel latches the timeout status.
#pragma once

#include <cuda.h>   // CUtensorMap (the tensor map is encoded on the host)

#include "at_kernels.cuh"

namespace atk {

constexpr int kThreads3 = 256;          // threads of a CTA (128 for groups of 4 columns)
constexpr int kMaxFields3 = 6;          // fields of the system (u, v, w and up to 3 scalars)
#ifndef AT_MIN_CTAS_3D
#define AT_MIN_CTAS_3D 2      // resident CTAs per SM the 3D stepper is compiled for
#endif

struct Params3 {
    void *u;
    unsigned char *ring;        // [T][P][6][face_words] words
    unsigned long long *flag;   // [P][6]
    int *ctrl;
    unsigned long long *hist;
    unsigned long long *gbar;
    int8_t *delays;             // [n_steps][P][6]
    long long n0, n1, n2;       // points per axis
    int m0, m1, m2;             // points per subdomain per axis
    long long P0, P1, P2, P;
    int L, T, mode, stages;
    int sb;                     // levels per pass (the blocked free-running stepper)
    int skip_publish;           // test knob: CTA 0 stops releasing flags beyond level skip_step
    long long skip_step;
    long long n_steps;
    unsigned long long seed;
    double cA[3], cB[3];        // dt / (2 dx_a), nu dt / dx_a^2
    double cBf[kMaxFields3][3]; // the system: kappa_f dt / dx_a^2 per field
    float cA32[3], cBf32[kMaxFields3][3];   // the same, rounded to FP32 once on the host
    int nf;                     // fields (1: the scalar equation)
    long long face_words;       // words per field of a ring entry (a multiple of 4)
    int G;
    long long timeout_ns;
};

// shared memory: mbarriers, delay counters, per-tile face data, the six
// extrapolated halo planes of the tile (x faces [z][y], y faces [z][x], z
// faces [y][x]), plane stages
struct Smem3 {
    long long bar_off, hist_off, face_off, halo_off, halo_words[6], halo_at[6], stage_off, plane_bytes, total;
};

__host__ __device__ inline Smem3 smem3_layout(int m0, int m1, int m2, int word, int stages, int nf = 1)
{
    Smem3 l;
    l.bar_off = 0;                                   // full[stages], then two ints per stage
    l.hist_off = round_up(16LL * stages, 16);
    l.face_off = round_up(l.hist_off + 4LL * (kMaxL + 1), 16);
    l.halo_off = round_up(l.face_off + 6 * 16 + 16, 128);
    long long at = l.halo_off;
    for (int f = 0; f < 6; ++f) {                    // per face: nf fields of halo_words each
        l.halo_words[f] = f < 2 ? (long long)m1 * m2 : f < 4 ? (long long)m0 * m2 : (long long)m0 * m1;
        l.halo_at[f] = at;
        at = round_up(at + (long long)nf * l.halo_words[f] * word, 16);
    }
    l.stage_off = round_up(at, 128);
    l.plane_bytes = round_up((long long)nf * m0 * m1 * word, 128);   // a plane of every field
    l.total = l.stage_off + (long long)stages * l.plane_bytes;
    return l;
}

static __device__ __noinline__ void raise_timeout3(const Params3 &p, int where, long long n, long long nb)
{
    if (atomicCAS(p.ctrl + kCtrlStatus, 0, kStatusTimeout) == 0) {
        p.ctrl[kCtrlCta] = (int)blockIdx.x;
        p.ctrl[kCtrlWhere] = where;
        p.ctrl[kCtrlNb] = (int)nb;
        p.ctrl[kCtrlStep] = (int)n;
    }
    atomicExch(p.ctrl + kCtrlAbort, 1);
}

static __device__ __noinline__ bool wait_flag3(const Params3 &p, const unsigned long long *fl, long long need,
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
            raise_timeout3(p, kWhereFlag, n, nb);
            return false;
        }
    }
}

// all threads wait (bounded) for the bulk copies into a stage
static __device__ __noinline__ bool wait_stage3(const Params3 &p, uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (ld_relaxed(p.ctrl + kCtrlAbort)) return false;
        if ((long long)(global_ns() - t0) > p.timeout_ns) {
            raise_timeout3(p, kWhereTile, -1, -1);
            return false;
        }
    }
}

// grid barrier before level `step` (1-based within the launch), one arrival
// per CTA; bounded.  Returns false on abort.
static __device__ __noinline__ bool grid_sync3(const Params3 &p, long long step, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(p.gbar, 1ull);
        const unsigned long long target = (unsigned long long)step * (unsigned long long)p.G;
        const unsigned long long t0 = global_ns();
        int ok = 1;
        while (ld_acquire(p.gbar) < target) {
            if (ld_relaxed(p.ctrl + kCtrlAbort)) { ok = 0; break; }
            if ((long long)(global_ns() - t0) > p.timeout_ns) { raise_timeout3(p, kWhereGrid, step, -1); ok = 0; break; }
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// neighbour of subdomain (p0, p1, p2) across face f
__device__ __forceinline__ long long face_neighbour(const Params3 &p, long long q0, long long q1, long long q2, int f)
{
    const int a = f >> 1, up = f & 1;
    if (a == 0) q0 = up ? (q0 + 1 == p.P0 ? 0 : q0 + 1) : (q0 == 0 ? p.P0 - 1 : q0 - 1);
    else if (a == 1) q1 = up ? (q1 + 1 == p.P1 ? 0 : q1 + 1) : (q1 == 0 ? p.P1 - 1 : q1 - 1);
    else q2 = up ? (q2 + 1 == p.P2 ? 0 : q2 + 1) : (q2 == 0 ? p.P2 - 1 : q2 - 1);
    return (q2 * p.P1 + q1) * p.P0 + q0;
}

// ring entry of (level, subdomain, face): nf arrays of face_words words
template <typename T>
__device__ __forceinline__ T *ring_entry(const Params3 &p, long long level, long long sub, int face)
{
    return reinterpret_cast<T *>(p.ring) +
           (((size_t)(level & (p.T - 1)) * p.P + sub) * 6 + face) * (size_t)p.face_words * (size_t)p.nf;
}

// NF fields stored one after another; SYS: the system of Eq. BS (fields 0, 1,
// 2 are the velocity (u, v, w), each field is advected by it and diffused with
// its own kappa); otherwise NF = 1 and the scalar equation
// u_t + u (u_x + u_y + u_z) = nu lap u.  A plane of every field arrives with
// one copy of a 4D tensor map (x, y, z, field).
// VW consecutive words (VW = 1 or 4; 16-byte aligned for 4) to global memory
template <typename T, int VW>
__device__ __forceinline__ void stv(T *g, const T *v)
{
    if constexpr (VW == 4 && sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(g) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int i = 0; i < VW; ++i) g[i] = v[i];
    }
}

// ISO (the scalar equation): equal spacing on the three axes, one
// coefficient pair, the six neighbours summed before scaling
template <typename T, int TC, int NF, bool SYS, int VW, int NT = kThreads3, bool ISO = false>
__global__ void __launch_bounds__(NT, NT == kThreads3 ? AT_MIN_CTAS_3D : 2 * AT_MIN_CTAS_3D)
    at_stepper3d(const Params3 p, const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const Smem3 sl = smem3_layout(p.m0, p.m1, p.m2, (int)sizeof(T), p.stages, NF);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + sl.bar_off);
    unsigned *hist = reinterpret_cast<unsigned *>(smem + sl.hist_off);
    int *s_flag = reinterpret_cast<int *>(smem + sl.face_off + 80);          // barrier / abort word
    unsigned char *stages = smem + sl.stage_off;
    // halo planes of face f, field q: halo_at[f] + q * halo_words[f] words
    T *hx0 = reinterpret_cast<T *>(smem + sl.halo_at[0]), *hx1 = reinterpret_cast<T *>(smem + sl.halo_at[1]);
    T *hy0 = reinterpret_cast<T *>(smem + sl.halo_at[2]), *hy1 = reinterpret_cast<T *>(smem + sl.halo_at[3]);
    T *hz0 = reinterpret_cast<T *>(smem + sl.halo_at[4]), *hz1 = reinterpret_cast<T *>(smem + sl.halo_at[5]);
    const int hwx = (int)sl.halo_words[0], hwy = (int)sl.halo_words[2], hwz = (int)sl.halo_words[4];
    const long long fw = p.face_words;

    const int tid = threadIdx.x, lane = tid & 31;
    const long long lo = (long long)blockIdx.x * p.P / p.G, hi = (long long)(blockIdx.x + 1) * p.P / p.G;
    const long long S = hi - lo;
    const long long lev0 = *reinterpret_cast<const volatile long long *>(p.ctrl + kCtrlN0);
    const int NS = p.stages;
    const int m0 = p.m0, m1 = p.m1, m2 = p.m2;
    const int PW = m0 * m1;
    const unsigned plane_bytes = (unsigned)(NF * PW * (int)sizeof(T));   // one box: a plane of every field
    const long long Q = p.n_steps * S * m2;                 // planes this CTA sweeps
    // (FP32: the host's FP32 copies, so no conversion is ever redone in the loop)
    constexpr bool F32 = sizeof(T) == 4;
    const T cA0 = F32 ? (T)p.cA32[0] : (T)p.cA[0], cA1 = F32 ? (T)p.cA32[1] : (T)p.cA[1],
            cA2 = F32 ? (T)p.cA32[2] : (T)p.cA[2];
    T cB[NF][3];
#pragma unroll
    for (int q = 0; q < NF; ++q) {
#pragma unroll
        for (int a = 0; a < 3; ++a) cB[q][a] = F32 ? (T)p.cBf32[SYS ? q : 0][a] : (T)(SYS ? p.cBf[q][a] : p.cB[a]);
    }
    T *u = reinterpret_cast<T *>(p.u);
    const long long field_words = p.n0 * p.n1 * p.n2;

    constexpr int kWarps3 = NT / 32;
    // per stage: warps done with its plane (the last one refills it), fills issued
    int *s_done = reinterpret_cast<int *>(bars + NS), *s_fills = s_done + NS;
    if (tid < NS) {
        mbar_init(&bars[tid], 1);
        s_done[tid] = 0;
        s_fills[tid] = 0;
    }
    if (tid == 0) { mbar_fence_init(); *s_flag = 0; }
    for (int i = tid; i <= kMaxL; i += NT) hist[i] = 0u;
    __syncthreads();

    // word offset of the first point of subdomain `sub` in u
    const long long plane_words = p.n0 * p.n1;
    // (subdomain indices in 32 bits: the host keeps P < 2^31, and a 64-bit
    // division costs tens of instructions on every thread of a tile start)
    const unsigned uP0 = (unsigned)p.P0, uP01 = (unsigned)(p.P0 * p.P1);
    auto tile_base = [&](long long sub) -> long long {
        const unsigned us = (unsigned)sub, q2 = us / uP01, r = us - q2 * uP01, q1 = r / uP0, q0 = r - q1 * uP0;
        return ((long long)q2 * m2) * plane_words + ((long long)q1 * m1) * p.n0 + (long long)q0 * m0;
    };
    // element coordinates of the first point of subdomain `sub`
    auto tile_coords = [&](long long sub, int *x, int *y, int *z) {
        const unsigned us = (unsigned)sub, q2 = us / uP01, r = us - q2 * uP01, q1 = r / uP0, q0 = r - q1 * uP0;
        *x = (int)(q0 * m0); *y = (int)(q1 * m1); *z = (int)(q2 * m2);
    };
    // one plane of every field into stage st (lane 0 of the issuing warp)
    auto issue_plane = [&](int st, int x0, int y0, int z0) {
        mbar_arrive_expect_tx(&bars[st], plane_bytes);
        tensor_load_4d(stages + (size_t)st * sl.plane_bytes, &tmap, x0, y0, z0, 0, &bars[st]);
        ++s_fills[st];
    };
    // element coordinates of the current tile's subdomain and of the next
    // tile's (a refill is at most stages <= m2 planes ahead)
    int tx0, ty0, tz0, nx0, ny0, nz0;
    tile_coords(lo, &tx0, &ty0, &tz0);
    tile_coords(lo + 1 == hi ? lo : lo + 1, &nx0, &ny0, &nz0);

    // column groups of this thread: first column, offset in a plane of u,
    // faces touched (x: by the group's first / last column)
    int cx[TC], cy[TC], coff[TC], cface[TC];
    bool cv[TC];
    const int GR = m0 / VW;                  // groups per row (the host checks VW | m0)
#pragma unroll
    for (int q = 0; q < TC; ++q) {
        const int c = tid + NT * q;
        cv[q] = c < PW / VW;
        cx[q] = cv[q] ? (c % GR) * VW : 0;
        cy[q] = cv[q] ? c / GR : 0;
        coff[q] = cy[q] * (int)p.n0 + cx[q];
        cface[q] = (cx[q] == 0 ? 1 : 0) | (cx[q] + VW == m0 ? 2 : 0) | (cy[q] == 0 ? 4 : 0) | (cy[q] == m1 - 1 ? 8 : 0);
    }
    T prev[NF][TC][VW], cur[NF][TC][VW];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int q = 0; q < TC; ++q)
#pragma unroll
            for (int e = 0; e < VW; ++e) prev[f][q][e] = cur[f][q][e] = (T)0;

    if (tid == 0)
        for (int st = 0; st < NS && st < Q; ++st) issue_plane(st, tx0, ty0, tz0 + st);
    // a failed wait is recorded in s_flag; every thread acts on it at the
    // next CTA barrier (at a tile start), so control flow stays uniform there.
    // Planes are consumed in order: gs, gp are the stage and fill parity of
    // the current plane g (running counters: no division per plane).
    int gs = 0;
    unsigned gp = 0;
    // Lane 0 of each warp waits and the warp follows it (warp-uniform
    // outcome: the plane loop exchanges words by shuffles).
    auto wait_plane = [&](int st, unsigned par) -> bool {
        int good = 1;
        if (lane == 0 && !mbar_try_wait(&bars[st], par)) good = wait_stage3(p, &bars[st], par) ? 1 : 0;
        good = __shfl_sync(0xffffffffu, good, 0);
        __syncwarp();
        if (!good) { if (lane == 0) atomicExch(s_flag, -1); return false; }
        return true;
    };

    // Every warp runs the same number of tiles and meets the same CTA
    // barriers; a failed wait inside a tile only skips that warp's remaining
    // planes, and all threads leave together after the next tile-start barrier.
    bool ok = true;
    long long lv = lev0, sub = lo;
    long long g = 0;                         // plane of the sweep being computed (0 .. Q-1)
    long long prev_sub = -1, prev_new = 0;   // the tile whose flags are still to be released
    T *rf[6];                                // ring entries of the new level of the current tile
    const long long n_tiles = p.n_steps * S;
    for (long long t = 0; t < n_tiles; ++t) {
        // ---- tile start (two CTA barriers): release the previous tile's
        // flags, grid barrier (synchronous mode), delays, halos
        __syncthreads();
        if (*s_flag == -1) { ok = false; break; }
        if (tid == 0 && prev_sub >= 0 && !(p.skip_publish && blockIdx.x == 0 && prev_new > p.skip_step)) {
            __threadfence();
            for (int f = 0; f < 6; ++f) st_release(p.flag + prev_sub * 6 + f, (unsigned long long)prev_new);
        }
        if (p.mode == kModeSync && sub == lo && lv > lev0) {
            if (!grid_sync3(p, lv - lev0, s_flag)) { ok = false; break; }
        }
        const unsigned us = (unsigned)sub, us2 = us / uP01, usr = us - us2 * uP01, us1 = usr / uP0;
        const long long s0 = usr - us1 * uP0, s1 = us1, s2 = us2;
        const long long base = tile_base(sub);
#pragma unroll
        for (int f = 0; f < 6; ++f) rf[f] = ring_entry<T>(p, lv + 1, sub, f);
        // warp w takes faces w, w + NT/32, ... (< 6): its lane 0 chooses the
        // delay and checks (or waits for) the neighbour's flag, then the warp
        // stages the face's halo plane -- the neighbour's facing ring
        // entries, extrapolated once with the delay (16-byte loads where aligned)
        for (int f = tid >> 5; f < 6; f += kWarps3) {
            const long long q = face_neighbour(p, s0, s1, s2, f);
            long long k = 0;
            int good = 1;
            if (lane == 0) {
                long long kmax = lv - 2 + 1;           // s = 2 levels per extrapolation
                if (kmax < 0) kmax = 0;
                if (kmax > p.L) kmax = p.L;
                if (p.mode == kModeSeeded) {
                    const unsigned long long ctr = ((unsigned long long)lv * (unsigned long long)p.P +
                                                    (unsigned long long)sub) * 6ull + (unsigned long long)f;
                    k = (long long)(((splitmix64(p.seed, ctr) >> 32) * (unsigned long long)(p.L + 1)) >> 32);
                } else if (p.mode == kModeReplay) {
                    k = p.delays[((size_t)(lv - lev0) * p.P + sub) * 6 + f];
                }
                if (k > kmax) k = kmax;
                if (k < 0) k = 0;
                if (p.mode != kModeSync) {
                    const unsigned long long *fl = p.flag + q * 6 + (f ^ 1);
                    const long long need = (p.mode == kModeFree) ? lv - kmax : lv - k;
                    unsigned long long seen = ld_acquire(fl);
                    if ((long long)seen < need && !wait_flag3(p, fl, need, &seen, lv, q)) good = 0;
                    if (good && p.mode == kModeFree) k = lv - ((long long)seen < lv ? (long long)seen : lv);
                }
                if (good) {
                    atomicAdd(&hist[k], 1u);
                    if (p.delays && p.mode != kModeReplay)
                        p.delays[((size_t)(lv - lev0) * p.P + sub) * 6 + f] = (int8_t)k;
                } else {
                    atomicExch(s_flag, -1);
                }
            }
            good = __shfl_sync(0xffffffffu, good, 0);
            const int kk = __shfl_sync(0xffffffffu, (int)k, 0);
            if (good) {
                const T *e0 = ring_entry<T>(p, lv - kk, q, f ^ 1);
                const T *e1 = ring_entry<T>(p, lv - kk - 1, q, f ^ 1);
                // (entries of the layout picked by selects: no local-memory copy)
                long long hat = sl.halo_at[0], hwd = sl.halo_words[0];
#pragma unroll
                for (int i = 1; i < 6; ++i) {
                    hat = f == i ? sl.halo_at[i] : hat;
                    hwd = f == i ? sl.halo_words[i] : hwd;
                }
                T *h = reinterpret_cast<T *>(smem + hat);
                const int nw = (int)hwd;
                // (k+1) f0 - k f1 in Newton form f0 + k (f0 - f1): the difference
                // of nearby levels is exact, so the rounding stays about an ulp
                const T b = (T)kk;
                for (int fld = 0; fld < NF; ++fld) {
                    const T *s0p = e0 + fld * fw, *s1p = e1 + fld * fw;
                    T *hp = h + fld * nw;
                    if (sizeof(T) == 4 && (nw & 3) == 0) {
                        for (int i = 4 * lane; i < nw; i += 128) {
                            T v0[4], v1[4];
                            lds<T, 4>(s0p + i, v0);           // (a 16-byte generic load of global memory)
                            if (kk != 0) {
                                lds<T, 4>(s1p + i, v1);
#pragma unroll
                                for (int e = 0; e < 4; ++e) v0[e] = v0[e] + b * (v0[e] - v1[e]);
                            }
                            sts4<T>(hp + i, v0);
                        }
                    } else {
                        for (int i = lane; i < nw; i += 32)
                            hp[i] = kk == 0 ? s0p[i] : s0p[i] + b * (s0p[i] - s1p[i]);
                    }
                }
            }
        }
        if (tid == 0 && p.mode == kModeSync) __threadfence();
        __syncthreads();
        if (*s_flag == -1) { ok = false; break; }
        // plane z = -1 (the -z halo) and plane 0
        if (!wait_plane(gs, gp)) { ok = false; }
        {
            const T *st0 = reinterpret_cast<const T *>(stages + (size_t)gs * sl.plane_bytes);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
#pragma unroll
                for (int q = 0; q < TC; ++q) {
                    if (!cv[q]) continue;
                    lds<T, VW>(hz0 + f * hwz + cy[q] * m0 + cx[q], prev[f][q]);
                    lds<T, VW>(st0 + f * PW + cy[q] * m0 + cx[q], cur[f][q]);
                }
            }
        }
        const long long lnew = lv + 1;
        // ---- the planes of the tile; warps run independently (stage
        // barriers only)
        for (int z = 0; z < m2 && ok; ++z) {
            const bool top = (z == m2 - 1);
            const int sg = gs, sg1 = gs + 1 == NS ? 0 : gs + 1;
            const unsigned gp1 = sg1 == 0 ? gp ^ 1u : gp;
            if (!top && !wait_plane(sg1, gp1)) { ok = false; break; }
            const T *st = reinterpret_cast<const T *>(stages + (size_t)sg * sl.plane_bytes);
            const T *stn = reinterpret_cast<const T *>(stages + (size_t)sg1 * sl.plane_bytes);
            T *up = u + base + (long long)z * plane_words;
            const int zy = z * m1, zx = z * m0;
#pragma unroll
            for (int q = 0; q < TC; ++q) {
                if (VW == 1 && !cv[q]) continue;            // groups of 4: every thread has one
                const int x = cx[q], y = cy[q], c = y * m0 + x;
                const int fc = cface[q];
                // advecting velocity at the points, level n (the system)
                T Uv[VW], Vv[VW], Wv[VW];
#pragma unroll
                for (int e = 0; e < VW; ++e) {
                    Uv[e] = SYS ? cur[0][q][e] : (T)0;
                    Vv[e] = SYS ? cur[1 % NF][q][e] : (T)0;
                    Wv[e] = SYS ? cur[2 % NF][q][e] : (T)0;
                }
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const T *sf = st + f * PW;
                    T ab[VW], ym[VW], yp[VW], un[VW];
                    lds<T, VW>(top ? hz1 + f * hwz + c : stn + f * PW + c, ab);
                    lds<T, VW>((fc & 4) ? hy0 + f * hwy + zx + x : sf + c - m0, ym);
                    lds<T, VW>((fc & 8) ? hy1 + f * hwy + zx + x : sf + c + m0, yp);
                    T xl, xr;
                    if constexpr (VW == 4) {
                        // a row is GR <= 32 consecutive lanes of one warp: the
                        // words beyond the group are the neighbouring lanes'
                        const T lft = __shfl_up_sync(0xffffffffu, cur[f][q][VW - 1], 1);
                        const T rgt = __shfl_down_sync(0xffffffffu, cur[f][q][0], 1);
                        xl = (fc & 1) ? hx0[f * hwx + zy + y] : lft;
                        xr = (fc & 2) ? hx1[f * hwx + zy + y] : rgt;
                    } else {
                        xl = (fc & 1) ? hx0[f * hwx + zy + y] : sf[c - 1];
                        xr = (fc & 2) ? hx1[f * hwx + zy + y] : sf[c + VW];
                    }
#pragma unroll
                    for (int e = 0; e < VW; ++e) {
                        const T cc = cur[f][q][e], below = prev[f][q][e], above = ab[e];
                        const T xm = e == 0 ? xl : cur[f][q][e > 0 ? e - 1 : 0];
                        const T xp = e == VW - 1 ? xr : cur[f][q][e + 1 < VW ? e + 1 : e];
                        const T d2 = cB[f][0] * ((xp + xm) - (T)2 * cc) + cB[f][1] * ((yp[e] + ym[e]) - (T)2 * cc) +
                                     cB[f][2] * ((above + below) - (T)2 * cc);
                        if constexpr (SYS) {
                            const T adv = cA0 * Uv[e] * (xp - xm) + cA1 * Vv[e] * (yp[e] - ym[e]) +
                                          cA2 * Wv[e] * (above - below);
                            un[e] = cc + (d2 - adv);
                        } else if constexpr (ISO) {
                            const T sum = ((xp + xm) + (yp[e] + ym[e])) + (above + below);
                            const T dif = ((xp - xm) + (yp[e] - ym[e])) + (above - below);
                            un[e] = cc + (cB[f][0] * (sum - (T)6 * cc) - cc * (cA0 * dif));
                        } else {
                            const T d1 = cA0 * (xp - xm) + cA1 * (yp[e] - ym[e]) + cA2 * (above - below);
                            un[e] = cc + (d2 - cc * d1);
                        }
                    }
                    stv<T, VW>(up + f * field_words + coff[q], un);
                    // boundary values of the new level into the ring
                    if (fc) {
                        if (fc & 1) rf[0][f * fw + zy + y] = un[0];
                        if (fc & 2) rf[1][f * fw + zy + y] = un[VW - 1];
                        if (fc & 4) stv<T, VW>(rf[2] + f * fw + zx + x, un);
                        if (fc & 8) stv<T, VW>(rf[3] + f * fw + zx + x, un);
                    }
                    if (z == 0) stv<T, VW>(rf[4] + f * fw + c, un);
                    if (top) stv<T, VW>(rf[5] + f * fw + c, un);
#pragma unroll
                    for (int e = 0; e < VW; ++e) {
                        prev[f][q][e] = cur[f][q][e];
                        cur[f][q][e] = ab[e];
                    }
                }
            }
            // the next read of a plane written here is a bulk copy (async
            // proxy) at the next level: with two or more subdomains per CTA it
            // is issued after this tile ends, so one proxy fence per tile (it
            // waits for this thread's stores) covers every plane; with one
            // subdomain, fence every plane
            if (top || S == 1) fence_proxy_async_global();
            __syncwarp();
            // done with stage sg (plane g; plane g - 1 read it as the plane
            // above): the last warp refills it with plane g + NS
            if (lane == 0) {
                __threadfence_block();
                if (atomicAdd(&s_done[sg], 1) == kWarps3 - 1) {
                    s_done[sg] = 0;
                    __threadfence_block();
                    if (g + NS < Q) {
                        if (z + NS < m2) issue_plane(sg, tx0, ty0, tz0 + z + NS);
                        else issue_plane(sg, nx0, ny0, nz0 + z + NS - m2);
                    }
                }
            }
            ++g;
            gs = sg1;
            gp = gp1;
        }
        prev_sub = sub;
        prev_new = lnew;
        if (++sub == hi) { sub = lo; ++lv; }
        // coordinates of the new tile and of the one after it
        tx0 = nx0; ty0 = ny0; tz0 = nz0;
        tile_coords(sub + 1 == hi ? lo : sub + 1, &nx0, &ny0, &nz0);
    }
    __syncthreads();
    if (tid == 0 && ok && prev_sub >= 0 && !(p.skip_publish && blockIdx.x == 0 && prev_new > p.skip_step)) {
        __threadfence();
        for (int f = 0; f < 6; ++f) st_release(p.flag + prev_sub * 6 + f, (unsigned long long)prev_new);
    }
    // let the copies in flight land before leaving (the latest fill of each
    // stage completes the phase of parity (fills - 1) & 1)
    if (tid == 0) {
        for (int st = 0; st < NS; ++st) {
            if (s_fills[st] == 0) continue;
            const unsigned par = (unsigned)((s_fills[st] - 1) & 1);
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(&bars[st], par) && (long long)(global_ns() - t0) < p.timeout_ns) {
            }
        }
    }
    __syncthreads();
    if (tid <= p.L && tid <= kMaxL && hist[tid]) atomicAdd(p.hist + tid, (unsigned long long)hist[tid]);
    (void)ok;
    // the last CTA to finish advances the level and rearms the grid barrier
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(p.ctrl + kCtrlDone, 1) == p.G - 1) {
            *reinterpret_cast<volatile long long *>(p.ctrl + kCtrlN0) = lev0 + p.n_steps;
            *reinterpret_cast<volatile int *>(p.ctrl + kCtrlDone) = 0;
            *reinterpret_cast<volatile unsigned long long *>(p.gbar) = 0ull;
            __threadfence();
        }
    }
}

// level-0 ring entries of every face, flags and control block
template <typename T>
__global__ void at_init3d(const Params3 p)
{
    const int PWmax = (int)p.face_words;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long total = p.P * 6 * p.nf * PWmax;
    const long long field_words = p.n0 * p.n1 * p.n2;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const long long sub = t / (6 * p.nf * PWmax);
        const int f = (int)((t / ((long long)p.nf * PWmax)) % 6);
        const int fld = (int)((t / PWmax) % p.nf);
        const int e = (int)(t % PWmax);
        const T *u = reinterpret_cast<const T *>(p.u) + (size_t)fld * field_words;
        const long long s0 = sub % p.P0, s1 = (sub / p.P0) % p.P1, s2 = sub / (p.P0 * p.P1);
        int x, y, z;
        if (f < 2) {            // [z][y]
            if (e >= p.m1 * p.m2) continue;
            z = e / p.m1; y = e % p.m1; x = f == 0 ? 0 : p.m0 - 1;
        } else if (f < 4) {     // [z][x]
            if (e >= p.m0 * p.m2) continue;
            z = e / p.m0; x = e % p.m0; y = f == 2 ? 0 : p.m1 - 1;
        } else {                // [y][x]
            if (e >= p.m0 * p.m1) continue;
            y = e / p.m0; x = e % p.m0; z = f == 4 ? 0 : p.m2 - 1;
        }
        const size_t gi = ((size_t)(s2 * p.m2 + z) * p.n1 + (size_t)(s1 * p.m1 + y)) * p.n0 + (size_t)(s0 * p.m0 + x);
        ring_entry<T>(p, 0, sub, f)[(size_t)fld * PWmax + e] = u[gi];
        if (e == 0 && fld == 0) p.flag[sub * 6 + f] = 0ull;
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x < kCtrlWords) p.ctrl[threadIdx.x] = 0;
        if (threadIdx.x <= p.L) p.hist[threadIdx.x] = 0ull;
        if (threadIdx.x == 0) *p.gbar = 0ull;
    }
}

}  // namespace atk
