// at_adjoint.cuh -- discrete adjoint of the AT time step (reverse mode).
//
// One step takes lambda^{n+1} = dJ/du^{n+1} to lambda^n = dJ/du^n for a
// scalar J of the final level, given the stored level u^n, the levels the
// delayed halos of level n were extrapolated from, and the delays of level n.
// One cooperative launch takes the steps of a whole checkpoint interval,
// n_hi - 1 down to n_lo, with a grid barrier (bounded) between steps.
//
// The forward step (Sec. 3.2, Eq. BS, AT halos of Eq. AT1/AT2 in split form)
// writes u^{n+1}_i = v_0 + cB b(v) - cA v_0 a(v) (+ forcing, independent of u
// and nu), with a = sum_j alpha_j v_j, b = sum_j beta_j v_j over the stencil
// values v_j (j = -R..R) of point i.  Each v_j is u^n at a point of the same
// subdomain, or across a subdomain face with delay k the extrapolation
// sum_m w_m(k) u^{n-k-m} of the neighbour's point.  So
//     d u^{n+1}_i / d v_j = [j = 0] (1 - cA a) + cB beta_j - cA v_0 alpha_j,
//     d u^{n+1}_i / d nu  = (cB / nu) b.
// lambda^n_i gathers, over every point r whose stencil reads u^n_i at level n
// (the point itself, its neighbours in the subdomain, and a neighbouring
// subdomain's boundary points when that face's delay is 0), the term
// lambda^{n+1}_r d u^{n+1}_r / d v_{i-r}.  Reads of older levels (k + m >= 1)
// are scattered into a pending ring [slot][P][2][R] by the one thread that owns
// the reading face (one writer per slot entry and step) and collected, then
// cleared, when the sweep reaches that level (no atomics there); dJ/dnu is
// summed per block in FP64 and added into the block's own slot (one add per
// block and launch, so the sum's order is fixed).  Blocks walk the subdomains, 4 points per thread; the
// word offsets of the levels read are computed on the host.
#pragma once

#include "at_device.cuh"

namespace atk {

constexpr int kAdjMaxLevels = 20;   // levels n .. n-L-s+1 a step reads (L <= 16, s <= 3)

struct AdjParams {
    const void *levels;        // full fields of the stored levels, N words each: level l in slot l mod Dl
    long long Dl;
    void *lam_a, *lam_b;       // lambda, N words each: lambda^{n_hi} in lam_a, then alternating
    void *pend;                // [Tp][P][2][R] words: adjoint of boundary values at older levels
    double *dnu_part;          // [gridDim.x * gridDim.y] running FP64 sums of dJ/dnu
    const int8_t *delays;      // delays of level n at delays[(n - k_level) * P * 2 + p * 2 + face]
    long long k_level;         // level of the delays' first row
    long long N, P, M;
    int L, Tp;                 // Tp: a power of two
    double cA, cB, dtdx2;      // as the stepper's; dtdx2 = cB / nu
    float cAf, cBf, dtdx2f;    // the same in FP32 (FP32 kernels convert nothing per point)
    long long n_hi, n_lo;      // this launch: lambda^{n_hi} -> lambda^{n_lo}, n_hi > n_lo
    unsigned long long *bar;   // grid-barrier arrivals, zero at the launch
    int *ctrl;                 // the solver's control block (status, abort word)
    long long timeout_ns;      // bound of each grid-barrier wait
};

template <int ORDER>
struct Coeffs;
template <>
struct Coeffs<2> {
    static __device__ __forceinline__ int alpha(int j) { return j; }                 // a = v1 - v-1
    static __device__ __forceinline__ int beta(int j) { return j == 0 ? -2 : 1; }    // b = v1 + v-1 - 2 v0
};
template <>
struct Coeffs<4> {
    // a = 8 (v1 - v-1) - (v2 - v-2), b = 16 (v1 + v-1) - (v2 + v-2) - 30 v0
    static __device__ __forceinline__ int alpha(int j) { return j == 0 ? 0 : (j == 1 ? 8 : j == -1 ? -8 : j == 2 ? -1 : 1); }
    static __device__ __forceinline__ int beta(int j) { return j == 0 ? -30 : (j == 1 || j == -1) ? 16 : -1; }
};

// Per-step view of the stored levels and the adjoint fields, with 32-bit
// indices within a level (the host checks N < 2^31); off[q] is the word
// offset of level n - q in the stored levels (in shared memory).
template <typename T, int ORDER>
struct AdjStep {
    static constexpr int R = ORDER / 2;
    static constexpr int S_LEV = ORDER / 2 + 1;
    const AdjParams &a;
    long long n;               // level of the lambda being computed
    const long long *off;
    const T *lev;              // stored levels
    const T *un;               // level n
    const T *lam;              // lambda^{n+1}
    int M, P;
    T cA, cB;

    __device__ AdjStep(const AdjParams &p, long long n_, const long long *off_, const T *lam_)
        : a(p), n(n_), off(off_), lev(reinterpret_cast<const T *>(p.levels)),
          un(reinterpret_cast<const T *>(p.levels) + off_[0]), lam(lam_), M((int)p.M), P((int)p.P)
    {
        if constexpr (sizeof(T) == 4) { cA = p.cAf; cB = p.cBf; }
        else { cA = (T)p.cA; cB = (T)p.cB; }
    }

    // delay of face f of subdomain p at level n (the forward run's, read from
    // the recomputation's record or the replayed array), clamped as the
    // forward run clamps it (no level below 0, at most L)
    __device__ int delay(int p, int f) const
    {
        int k = a.delays[((size_t)(n - a.k_level) * a.P + p) * 2 + f];
        long long kmax = n - S_LEV + 1;
        if (kmax < 0) kmax = 0;
        if (kmax > a.L) kmax = a.L;
        if (k > kmax) k = (int)kmax;
        if (k < 0) k = 0;
        return k;
    }

    // halo value of point src extrapolated with delay k (same operations as
    // the stepper's halo approximation: Newton form)
    __device__ T halo(int src, int k) const
    {
        const T r0 = lev[off[k] + src];
        if (k == 0) return r0;
        const T r1 = lev[off[k + 1] + src];
        const T d1 = r0 - r1;
        if constexpr (S_LEV == 2) {
            return r0 + (T)k * d1;
        } else {
            const T r2 = lev[off[k + 2] + src];
            const T d2 = d1 - (r1 - r2);
            return r0 + ((T)k * d1 + (T)(k * (k + 1) / 2) * d2);
        }
    }

    __device__ int left(int p) const { return p == 0 ? P - 1 : p - 1; }
    __device__ int right(int p) const { return p == P - 1 ? 0 : p + 1; }

    // stencil values v[0..2R] at level n of point loc of subdomain p, whose
    // faces have delays k0, k1
    __device__ void values(int p, int loc, int k0, int k1, T *v) const
    {
#pragma unroll
        for (int j = -R; j <= R; ++j) {
            const int lj = loc + j;
            if (lj < 0) v[j + R] = halo(left(p) * M + M + lj, k0);
            else if (lj >= M) v[j + R] = halo(right(p) * M + (lj - M), k1);
            else v[j + R] = un[p * M + lj];
        }
    }

    // lambda^{n+1}_r d u^{n+1}_r / d v_j, given the values v of point r
    __device__ T gbar(int r, int j, const T *v) const
    {
        T av = (T)0;
#pragma unroll
        for (int q = -R; q <= R; ++q) av += (T)Coeffs<ORDER>::alpha(q) * v[q + R];
        T d = cB * (T)Coeffs<ORDER>::beta(j) - cA * v[R] * (T)Coeffs<ORDER>::alpha(j);
        if (j == 0) d += (T)1 - cA * av;
        return lam[r] * d;
    }

    __device__ T *pend(long long l, int p, int side, int r) const
    {
        return reinterpret_cast<T *>(a.pend) + (((size_t)(l & (a.Tp - 1)) * a.P + p) * 2 + side) * R + r;
    }
};

// Block (x, y) handles the chunk of points y*C .. y*C+C-1 (C = 1024: a thread
// takes 4 points, 256 apart) of subdomains x, x + gridDim.x, ...  Each point
// first computes the 2R+1 terms it contributes to the adjoint of its stencil
// values (c_j = lambda^{n+1}_r d u^{n+1}_r / d v_j) into shared memory; each
// point then gathers the terms of its readers from there.
constexpr int kAdjThreads = 256;
constexpr int kAdjPts = 4;                            // points per thread
constexpr int kAdjChunk = kAdjThreads * kAdjPts;      // points per block and subdomain

// One step, lambda^{n+1} (lam_in) -> lambda^n (lam_out), by this block;
// returns the block's FP64 contribution to dJ/dnu (thread 0).
template <typename T, int ORDER>
__device__ double adjoint_level(const AdjParams &a, long long n, const long long *s_off, const T *lam_in, T *lam_out,
                                T (*s_c)[kAdjChunk], T *red)
{
    constexpr int R = ORDER / 2;
    constexpr int S_LEV = ORDER / 2 + 1;
    const AdjStep<T, ORDER> A(a, n, s_off, lam_in);
    T nu_acc = (T)0;          // this thread's sum of lambda^{n+1}_i b_i
    const T dtdx2 = sizeof(T) == 4 ? (T)a.dtdx2f : (T)a.dtdx2;
    const int tid = threadIdx.x, lane = tid & 31;
    const int M = A.M;
    const int chunk_lo = blockIdx.y * kAdjChunk;
    for (int p = blockIdx.x; p < A.P; p += gridDim.x) {
        const int pl = A.left(p), pr = A.right(p);
        // loads that need no delay first (lambda^{n+1}; the pending words
        // addressed to this level), so that their latency overlaps the delays'
        T gl[kAdjPts], pw[kAdjPts];
#pragma unroll
        for (int kp = 0; kp < kAdjPts; ++kp) {
            const int loc = chunk_lo + tid + kp * kAdjThreads;
            gl[kp] = loc < M ? A.lam[p * M + loc] : (T)0;
            pw[kp] = loc < R ? *A.pend(n, p, 0, loc) : (loc >= M - R && loc < M) ? *A.pend(n, p, 1, loc - (M - R)) : (T)0;
        }
        // delays (lanes 0..3, then shared across the warp): this subdomain's
        // faces 0, 1; the left neighbour's face 1; the right neighbour's face 0
        int kk = 0;
        if (lane < 4) kk = A.delay(lane < 2 ? p : (lane == 2 ? pl : pr), lane < 2 ? lane : (lane == 2 ? 1 : 0));
        const int k0 = __shfl_sync(0xffffffffu, kk, 0), k1 = __shfl_sync(0xffffffffu, kk, 1);
        const int kl1 = __shfl_sync(0xffffffffu, kk, 2), kr0 = __shfl_sync(0xffffffffu, kk, 3);
        if (p != (int)blockIdx.x) __syncthreads();   // the previous subdomain's terms have been read
#pragma unroll
        for (int kp = 0; kp < kAdjPts; ++kp) {
            const int off = tid + kp * kAdjThreads, loc = chunk_lo + off;
            if (loc >= M) continue;
            T v[2 * R + 1];
            A.values(p, loc, k0, k1, v);
            T av = (T)0, bv = (T)0;
#pragma unroll
            for (int q = -R; q <= R; ++q) {
                av += (T)Coeffs<ORDER>::alpha(q) * v[q + R];
                bv += (T)Coeffs<ORDER>::beta(q) * v[q + R];
            }
            const T g = gl[kp];
#pragma unroll
            for (int j = -R; j <= R; ++j) {
                T d = A.cB * (T)Coeffs<ORDER>::beta(j) - A.cA * v[R] * (T)Coeffs<ORDER>::alpha(j);
                if (j == 0) d += (T)1 - A.cA * av;
                s_c[j + R][off] = g * d;
            }
            nu_acc += g * bv;
        }
        __syncthreads();
#pragma unroll
        for (int kp = 0; kp < kAdjPts; ++kp) {
            const int off = tid + kp * kAdjThreads, loc = chunk_lo + off;
            if (loc >= M) continue;
            const int i = p * M + loc;
            T v[2 * R + 1];
            T acc = (T)0;
            // readers r = i + d whose value j = -d is u^n_i
#pragma unroll
            for (int d = -R; d <= R; ++d) {
                const int rl = loc + d;
                if (rl >= 0 && rl < M) {
                    if (rl >= chunk_lo && rl < chunk_lo + kAdjChunk) {
                        acc += s_c[-d + R][off + d];
                    } else {
                        A.values(p, rl, k0, k1, v);
                        acc += A.gbar(i + d, -d, v);
                    }
                } else if (rl < 0) {
                    // the left neighbour's last points read u^n_i across their
                    // face 1; only an undelayed read lands on level n (with
                    // M >= 2R their stencils do not reach their own face 0)
                    if (kl1 == 0) {
                        A.values(pl, M + rl, -1, kl1, v);
                        acc += A.gbar(pl * M + M + rl, -d, v);
                    }
                } else if (kr0 == 0) {
                    A.values(pr, rl - M, kr0, -1, v);
                    acc += A.gbar(pr * M + (rl - M), -d, v);
                }
            }
            // delayed reads from later steps addressed to level n (loaded above)
            if (loc < R) {
                acc += pw[kp];
                *A.pend(n, p, 0, loc) = (T)0;
            } else if (loc >= M - R) {
                acc += pw[kp];
                *A.pend(n, p, 1, loc - (M - R)) = (T)0;
            }
            lam_out[i] = acc;

            // this subdomain's delayed reads across a face, scattered to older
            // levels of the neighbour's boundary values (one thread per face;
            // its readers are in its own chunk: the last chunk holds >= 4 points)
            if (loc == 0 || loc == M - 1) {
                const int f = loc == 0 ? 0 : 1;
                const int k = f == 0 ? k0 : k1;
                const int q = f == 0 ? pl : pr;
                T w[S_LEV];
                if constexpr (S_LEV == 2) {
                    w[0] = (T)(k + 1);
                    w[1] = (T)(-k);
                } else {
                    w[0] = (T)((k + 1) * (k + 2) / 2);
                    w[1] = (T)(-k * (k + 2));
                    w[2] = (T)(k * (k + 1) / 2);
                }
                // per source point of q: the sum of its readers' terms (source:
                // point M + t + j of q across face 0, j - t - 1 across face 1)
                T src[R];
#pragma unroll
                for (int r = 0; r < R; ++r) src[r] = (T)0;
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    const int rt = f == 0 ? off + t : off - t;         // reader's place in the chunk
#pragma unroll
                    for (int j = -R; j <= R; ++j) {
                        const bool crosses = f == 0 ? (j <= -t - 1) : (j >= t + 1);
                        if (!crosses) continue;
                        src[f == 0 ? R + t + j : j - t - 1] += s_c[j + R][rt];
                    }
                }
                // older levels n-k-m of those points: all loads, then all stores
                const int side = f == 0 ? 1 : 0;
                T old[S_LEV][R];
#pragma unroll
                for (int m = 0; m < S_LEV; ++m)
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        old[m][r] = (k + m == 0 || w[m] == (T)0) ? (T)0 : *A.pend(n - k - m, q, side, r);
#pragma unroll
                for (int m = 0; m < S_LEV; ++m) {
                    if (k + m == 0 || w[m] == (T)0) continue;     // level n: gathered above
#pragma unroll
                    for (int r = 0; r < R; ++r) *A.pend(n - k - m, q, side, r) = old[m][r] + w[m] * src[r];
                }
            }
        }
    }
    // dJ/dnu of this block: warp sums in the state's precision, then the
    // block's FP64 sum (one FP64 add per warp: FP64 is slow here)
    for (int o = 16; o > 0; o >>= 1) nu_acc += __shfl_xor_sync(0xffffffffu, nu_acc, o);
    if (lane == 0) red[tid >> 5] = nu_acc;
    __syncthreads();
    double sum = 0.0;
    if (tid == 0)
        for (int w = 0; w < kAdjThreads / 32; ++w) sum += (double)red[w] * (double)dtdx2;
    return sum;
}

// Grid barrier between the steps of an interval: every block arrives once
// per step (thread 0, after a block barrier and a fence) and waits for all;
// bounded by timeout_ns, after which the status and abort words are set and
// every block leaves.  Returns false on abort.
static __device__ __noinline__ bool adjoint_grid_sync(const AdjParams &a, unsigned long long target, long long n,
                                               int *s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.bar, 1ull);
        bool ok = true;
        if (ld_acquire(a.bar) < target) {
            const unsigned long long t0 = global_ns();
            for (;;) {
                __nanosleep(32);
                if (ld_acquire(a.bar) >= target) break;
                if (ld_relaxed(a.ctrl + kCtrlAbort)) { ok = false; break; }
                if ((long long)(global_ns() - t0) > a.timeout_ns) {
                    if (atomicCAS(a.ctrl + kCtrlStatus, 0, kStatusTimeout) == 0) {
                        a.ctrl[kCtrlCta] = (int)(blockIdx.y * gridDim.x + blockIdx.x);
                        a.ctrl[kCtrlWhere] = kWhereAdjoint;
                        a.ctrl[kCtrlNb] = -1;
                        a.ctrl[kCtrlStep] = (int)n;
                    }
                    atomicExch(a.ctrl + kCtrlAbort, 1);
                    ok = false;
                    break;
                }
            }
        }
        __threadfence();
        *s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

// The steps n_hi - 1 .. n_lo of one checkpoint interval in one cooperative
// launch (every block resident): lambda^{n_hi} in lam_a, lambda^{n_lo} in
// lam_a or lam_b after an even or odd number of steps.  Each block adds its
// dJ/dnu contribution of every step into its own FP64 running total, in the
// order of the steps.
template <typename T, int ORDER>
__global__ void __launch_bounds__(kAdjThreads, ORDER == 2 ? 7 : 3) at_adjoint_interval(const AdjParams a)
{
    constexpr int R = ORDER / 2;
    __shared__ T s_c[2 * R + 1][kAdjChunk];
    __shared__ T red[kAdjThreads / 32];
    __shared__ long long s_off[kAdjMaxLevels];
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    unsigned long long arrivals = 0;
    const unsigned long long nblocks = (unsigned long long)gridDim.x * gridDim.y;
    for (long long n = a.n_hi - 1, it = 0; n >= a.n_lo; --n, ++it) {
        // word offsets of the levels n, n-1, ..., n-L-s+1 in the stored ring
        if (tid < kAdjMaxLevels) s_off[tid] = (n - tid >= 0) ? ((n - tid) % a.Dl) * a.N : 0;
        __syncthreads();
        const T *lam_in = reinterpret_cast<const T *>((it & 1) ? a.lam_b : a.lam_a);
        T *lam_out = reinterpret_cast<T *>((it & 1) ? a.lam_a : a.lam_b);
        const double sum = adjoint_level<T, ORDER>(a, n, s_off, lam_in, lam_out, s_c, red);
        // one add per block and step into the block's own running total: a
        // reduction without return (no load on the block's critical path)
        if (tid == 0) atomicAdd(a.dnu_part + (size_t)blockIdx.y * gridDim.x + blockIdx.x, sum);
        if (n > a.n_lo) {
            arrivals += nblocks;
            if (!adjoint_grid_sync(a, arrivals, n, &s_ok)) return;
        }
    }
}

// ---------------------------------------------------------------------------
// The interval kernel for one subdomain per block (M <= kAdjOwnChunk points,
// every subdomain's block resident): a block keeps its own lambda in
// registers from level to level, and loads everything a level needs that does
// not depend on lambda -- the delays, its points' stencil values, the pending
// words its face threads will add to -- before the grid barrier that ends the
// previous level, so that after the barrier a level waits for one round trip
// at most (the neighbours' boundary lambdas and values, the pending words
// addressed to this level; edge threads only).  Same arithmetic, in the same
// order, as at_adjoint_interval.
constexpr int kAdjOwnThreads = 128;
constexpr int kAdjOwnPts = 8;                               // points per thread, kAdjOwnThreads apart
constexpr int kAdjOwnChunk = kAdjOwnThreads * kAdjOwnPts;

template <typename T, int ORDER>
__global__ void __launch_bounds__(kAdjOwnThreads, 7) at_adjoint_own(const AdjParams a)
{
    constexpr int R = ORDER / 2;
    constexpr int S_LEV = ORDER / 2 + 1;
    constexpr int NT = kAdjOwnThreads, PTS = kAdjOwnPts;
    __shared__ T s_c[2 * R + 1][kAdjOwnChunk];
    __shared__ T red[NT / 32];
    __shared__ long long s_off[2][kAdjMaxLevels];
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31;
    const int M = (int)a.M, P = (int)a.P;
    const int p = blockIdx.x;
    const int pl = p == 0 ? P - 1 : p - 1, pr = p == P - 1 ? 0 : p + 1;
    const T dtdx2 = sizeof(T) == 4 ? (T)a.dtdx2f : (T)a.dtdx2;
    // the face threads: point 0 (face 0) and point M-1 (face 1)
    const bool own_f0 = tid == 0, own_f1 = tid == (M - 1) % NT;
    const int kp_f1 = (M - 1) / NT;

    auto set_off = [&](long long n, int b) {
        if (tid < kAdjMaxLevels) s_off[b][tid] = (n - tid >= 0) ? ((n - tid) % a.Dl) * a.N : 0;
    };
    // extrapolation weights of a face with delay k
    auto weights = [&](int k, T *w) {
        if constexpr (S_LEV == 2) {
            w[0] = (T)(k + 1);
            w[1] = (T)(-k);
        } else {
            w[0] = (T)((k + 1) * (k + 2) / 2);
            w[1] = (T)(-k * (k + 2));
            w[2] = (T)(k * (k + 1) / 2);
        }
    };

    // what a level needs that does not depend on lambda
    T v[PTS][2 * R + 1];          // stencil values of this thread's points
    int k0 = 0, k1 = 0, kl1 = 0, kr0 = 0;
    T pold[2][S_LEV][R];          // face threads: current pending words of the levels they add to
    // (lanes 0..3: the raw delays of level n: this subdomain's faces 0, 1,
    // the left neighbour's face 1, the right neighbour's face 0 -- loaded a
    // level ahead, so that the prefetch below does not wait for them)
    auto load_delays = [&](long long n) -> int {
        const AdjStep<T, ORDER> A(a, n, s_off[0], nullptr);
        return lane < 4 ? A.delay(lane < 2 ? p : (lane == 2 ? pl : pr), lane < 2 ? lane : (lane == 2 ? 1 : 0)) : 0;
    };
    auto prefetch = [&](long long n, int b, int kk) {
        const AdjStep<T, ORDER> A(a, n, s_off[b], nullptr);
        k0 = __shfl_sync(0xffffffffu, kk, 0);
        k1 = __shfl_sync(0xffffffffu, kk, 1);
        kl1 = __shfl_sync(0xffffffffu, kk, 2);
        kr0 = __shfl_sync(0xffffffffu, kk, 3);
#pragma unroll
        for (int kp = 0; kp < PTS; ++kp) {
            const int loc = tid + kp * NT;
            if (loc < M) A.values(p, loc, k0, k1, v[kp]);
        }
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const bool mine = f == 0 ? own_f0 : own_f1;
            const int k = f == 0 ? k0 : k1;
            const int q = f == 0 ? pl : pr;
            T w[S_LEV];
            weights(k, w);
#pragma unroll
            for (int m = 0; m < S_LEV; ++m)
#pragma unroll
                for (int r = 0; r < R; ++r)
                    pold[f][m][r] = (mine && k + m != 0 && w[m] != (T)0) ? *A.pend(n - k - m, q, f == 0 ? 1 : 0, r)
                                                                         : (T)0;
        }
    };

    // lambda^{n_hi} of this block's points
    T lamr[PTS];
    {
        const T *l0 = reinterpret_cast<const T *>(a.lam_a);
#pragma unroll
        for (int kp = 0; kp < PTS; ++kp) {
            const int loc = tid + kp * NT;
            lamr[kp] = loc < M ? l0[(size_t)p * M + loc] : (T)0;
        }
    }
    set_off(a.n_hi - 1, 0);
    __syncthreads();
    prefetch(a.n_hi - 1, 0, load_delays(a.n_hi - 1));
    unsigned long long arrivals = 0;
    for (long long n = a.n_hi - 1, it = 0; n >= a.n_lo; --n, ++it) {
        const int b = (int)(it & 1);
        // the next level's delays and level offsets, early
        int kk_next = 0;
        if (n > a.n_lo) {
            kk_next = load_delays(n - 1);
            set_off(n - 1, b ^ 1);
        }
        const T *lam_in = reinterpret_cast<const T *>((it & 1) ? a.lam_b : a.lam_a);
        T *lam_out = reinterpret_cast<T *>((it & 1) ? a.lam_a : a.lam_b);
        const AdjStep<T, ORDER> A(a, n, s_off[b], lam_in);
        // the pending words addressed to this level (written by the
        // neighbours' face threads at later levels), loaded before any store
        // of the level: a thread holds at most one point within R of each face
        // The neighbours' readers across the faces (their lambda^{n+1} and
        // level-n values: an undelayed read lands on level n) likewise.
        T pwL = (T)0, pwR = (T)0, eL = (T)0, eR = (T)0;
        if (tid < R && tid < M) {
            pwL = *A.pend(n, p, 0, tid);
            if (kl1 == 0) {
#pragma unroll
                for (int d = -R; d < 0; ++d) {
                    const int rl = tid + d;
                    if (rl >= 0) continue;
                    T vv[2 * R + 1];
                    A.values(pl, M + rl, -1, kl1, vv);
                    eL += A.gbar(pl * M + M + rl, -d, vv);
                }
            }
        }
        {
            const int locR = tid + NT * ((M - 1 - tid) / NT);   // this thread's last point
            if (tid <= M - 1 && locR >= M - R && locR >= R) {
                pwR = *A.pend(n, p, 1, locR - (M - R));
                if (kr0 == 0) {
#pragma unroll
                    for (int d = 1; d <= R; ++d) {
                        const int rl = locR + d;
                        if (rl < M) continue;
                        T vv[2 * R + 1];
                        A.values(pr, rl - M, kr0, -1, vv);
                        eR += A.gbar(pr * M + (rl - M), -d, vv);
                    }
                }
            }
        }
        // terms c_j = lambda^{n+1}_r d u^{n+1}_r / d v_j of this block's points
        T nu_acc = (T)0;
#pragma unroll
        for (int kp = 0; kp < PTS; ++kp) {
            const int loc = tid + kp * NT;
            if (loc >= M) continue;
            T av = (T)0, bv = (T)0;
#pragma unroll
            for (int q = -R; q <= R; ++q) {
                av += (T)Coeffs<ORDER>::alpha(q) * v[kp][q + R];
                bv += (T)Coeffs<ORDER>::beta(q) * v[kp][q + R];
            }
            const T g = lamr[kp];
#pragma unroll
            for (int j = -R; j <= R; ++j) {
                T d = A.cB * (T)Coeffs<ORDER>::beta(j) - A.cA * v[kp][R] * (T)Coeffs<ORDER>::alpha(j);
                if (j == 0) d += (T)1 - A.cA * av;
                s_c[j + R][loc] = g * d;
            }
            nu_acc += g * bv;
        }
        __syncthreads();
        // gather lambda^n_i; the neighbours' readers across the faces from
        // their lambda^{n+1} and values (edge threads)
#pragma unroll
        for (int kp = 0; kp < PTS; ++kp) {
            const int loc = tid + kp * NT;
            if (loc >= M) continue;
            const int i = p * M + loc;
            T acc = (T)0;
#pragma unroll
            for (int d = -R; d <= R; ++d) {
                const int rl = loc + d;
                if (rl >= 0 && rl < M) acc += s_c[-d + R][rl];
            }
            // (the readers across the faces and the pending words, loaded
            // above; the words are then cleared)
            if (loc < R) acc += eL;
            if (loc >= M - R && loc >= R) acc += eR;
            if (loc < R) {
                acc += pwL;
                *A.pend(n, p, 0, loc) = (T)0;
            } else if (loc >= M - R) {
                acc += pwR;
                *A.pend(n, p, 1, loc - (M - R)) = (T)0;
            }
            lam_out[i] = acc;
            lamr[kp] = acc;
        }
        // this block's delayed reads across its faces, added to the
        // neighbours' boundary words at older levels (the face threads)
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            if (!(f == 0 ? own_f0 : own_f1)) continue;
            const int k = f == 0 ? k0 : k1;
            const int q = f == 0 ? pl : pr;
            const int off = f == 0 ? 0 : M - 1;
            T w[S_LEV];
            weights(k, w);
            T src[R];
#pragma unroll
            for (int r = 0; r < R; ++r) src[r] = (T)0;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int rt = f == 0 ? off + t : off - t;
#pragma unroll
                for (int j = -R; j <= R; ++j) {
                    const bool crosses = f == 0 ? (j <= -t - 1) : (j >= t + 1);
                    if (!crosses) continue;
                    src[f == 0 ? R + t + j : j - t - 1] += s_c[j + R][rt];
                }
            }
#pragma unroll
            for (int m = 0; m < S_LEV; ++m) {
                if (k + m == 0 || w[m] == (T)0) continue;     // level n: gathered above
#pragma unroll
                for (int r = 0; r < R; ++r) *A.pend(n - k - m, q, f == 0 ? 1 : 0, r) = pold[f][m][r] + w[m] * src[r];
            }
        }
        (void)kp_f1;
        // dJ/dnu: warp sums in the state's precision; thread 0 adds the
        // block's FP64 sum after the next block barrier
        for (int o = 16; o > 0; o >>= 1) nu_acc += __shfl_xor_sync(0xffffffffu, nu_acc, o);
        if (lane == 0) red[tid >> 5] = nu_acc;
        // the next level's lambda-free data (its loads land during the barrier)
        if (n > a.n_lo) prefetch(n - 1, b ^ 1, kk_next);
        __syncthreads();
        bool go = n > a.n_lo;
        if (tid == 0) {
            double sum = 0.0;
            for (int w = 0; w < NT / 32; ++w) sum += (double)red[w] * (double)dtdx2;
            atomicAdd(a.dnu_part + blockIdx.x, sum);
            if (go) {
                // grid barrier (bounded), as adjoint_grid_sync after its block barrier
                arrivals += gridDim.x;
                __threadfence();
                atomicAdd(a.bar, 1ull);
                bool ok = true;
                if (ld_acquire(a.bar) < arrivals) {
                    const unsigned long long t0 = global_ns();
                    for (;;) {
                        __nanosleep(32);
                        if (ld_acquire(a.bar) >= arrivals) break;
                        if (ld_relaxed(a.ctrl + kCtrlAbort)) { ok = false; break; }
                        if ((long long)(global_ns() - t0) > a.timeout_ns) {
                            if (atomicCAS(a.ctrl + kCtrlStatus, 0, kStatusTimeout) == 0) {
                                a.ctrl[kCtrlCta] = (int)blockIdx.x;
                                a.ctrl[kCtrlWhere] = kWhereAdjoint;
                                a.ctrl[kCtrlNb] = -1;
                                a.ctrl[kCtrlStep] = (int)n;
                            }
                            atomicExch(a.ctrl + kCtrlAbort, 1);
                            ok = false;
                            break;
                        }
                    }
                }
                __threadfence();
                s_ok = ok ? 1 : 0;
            }
        }
        if (go) {
            __syncthreads();
            if (!s_ok) return;
        }
    }
}

}  // namespace atk
