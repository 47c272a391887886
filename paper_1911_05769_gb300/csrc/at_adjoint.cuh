// at_adjoint.cuh -- discrete adjoint of the AT time step (reverse mode).
//
// One launch takes lambda^{n+1} = dJ/du^{n+1} to lambda^n = dJ/du^n for a
// scalar J of the final level, given the stored level u^n, the levels the
// delayed halos of level n were extrapolated from, and the delays of level n.
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
// cleared, when the sweep reaches that level.  No atomics; dJ/dnu is summed
// per block in FP64.
#pragma once

#include "at_device.cuh"

namespace atk {

struct AdjParams {
    const void *levels;        // u^l at slot l mod depth, N words each
    long long depth;
    const void *lam_in;        // lambda^{n+1}, N words
    void *lam_out;             // lambda^n, N words
    void *pend;                // [Tp][P][2][R] words: adjoint of boundary values at older levels
    double *dnu_part;          // [gridDim.x] running FP64 sums of dJ/dnu
    const int8_t *delays;      // replayed delays [levels][P][2], absolute level index
    long long N, P, M;
    int L, Tp, mode, per_sub;
    unsigned long long seed;
    double cA, cB, dtdx2;      // as the stepper's; dtdx2 = cB / nu
    long long n;               // level of lambda_out
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

template <typename T, int ORDER>
struct AdjStep {
    static constexpr int R = ORDER / 2;
    static constexpr int S_LEV = ORDER / 2 + 1;
    const AdjParams &a;

    __device__ T u(long long l, long long i) const
    {
        return reinterpret_cast<const T *>(a.levels)[(size_t)(l % a.depth) * (size_t)a.N + (size_t)i];
    }

    // delay of face f of subdomain p at level n, clamped as the forward run
    // clamps it (no level below 0, at most L)
    __device__ int delay(long long p, int f) const
    {
        int k = 0;
        if (a.mode == 1) k = seeded_delay(a.seed, a.n, p, a.P, a.per_sub ? 0 : f, a.L);
        else if (a.mode == 3) k = a.delays[((size_t)a.n * a.P + p) * 2 + f];
        long long kmax = a.n - S_LEV + 1;
        if (kmax < 0) kmax = 0;
        if (kmax > a.L) kmax = a.L;
        if (k > kmax) k = (int)kmax;
        if (k < 0) k = 0;
        return k;
    }

    // halo value of point src extrapolated with delay k (same operations as
    // the stepper's halo approximation)
    __device__ T halo(long long src, int k) const
    {
        const T r0 = u(a.n - k, src);
        if (k == 0) return r0;
        const T r1 = u(a.n - k - 1, src);
        if constexpr (S_LEV == 2) {
            return (T)(k + 1) * r0 - (T)k * r1;
        } else {
            const T r2 = u(a.n - k - 2, src);
            const T w0 = (T)((k + 1) * (k + 2) / 2);
            const T w1 = (T)(-k * (k + 2));
            const T w2 = (T)(k * (k + 1) / 2);
            return w0 * r0 + w1 * r1 + w2 * r2;
        }
    }

    // stencil values v[0..2R] of point r at level n
    __device__ void values(long long r, T *v) const
    {
        const long long p = r / a.M, loc = r - p * a.M;
        int kf[2] = {-1, -1};
#pragma unroll
        for (int j = -R; j <= R; ++j) {
            const long long lj = loc + j;
            if (lj >= 0 && lj < a.M) {
                v[j + R] = u(a.n, r + j);
            } else {
                const int f = lj < 0 ? 0 : 1;
                if (kf[f] < 0) kf[f] = delay(p, f);
                long long src = r + j;
                if (src < 0) src += a.N;
                if (src >= a.N) src -= a.N;
                v[j + R] = halo(src, kf[f]);
            }
        }
    }

    // lambda^{n+1}_r d u^{n+1}_r / d v_j, given the values v of point r
    __device__ T gbar(long long r, int j, const T *v) const
    {
        T av = (T)0;
#pragma unroll
        for (int q = -R; q <= R; ++q) av += (T)Coeffs<ORDER>::alpha(q) * v[q + R];
        const T g = reinterpret_cast<const T *>(a.lam_in)[r];
        T d = (T)a.cB * (T)Coeffs<ORDER>::beta(j) - (T)a.cA * v[R] * (T)Coeffs<ORDER>::alpha(j);
        if (j == 0) d += (T)1 - (T)a.cA * av;
        return g * d;
    }

    __device__ T *pend(long long l, long long p, int side, int r) const
    {
        return reinterpret_cast<T *>(a.pend) + (((size_t)(l % a.Tp) * a.P + p) * 2 + side) * R + r;
    }
};

template <typename T, int ORDER>
__global__ void __launch_bounds__(256) at_adjoint_step(const AdjParams a)
{
    constexpr int R = ORDER / 2;
    constexpr int S_LEV = ORDER / 2 + 1;
    const AdjStep<T, ORDER> A{a};
    double nu_acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += stride) {
        const long long p = i / a.M, loc = i - p * a.M;
        T v[2 * R + 1];
        T acc = (T)0;
        // readers r = i + d whose value j = -d is u^n_i
#pragma unroll
        for (int d = -R; d <= R; ++d) {
            const long long rl = loc + d;
            long long r = i + d;
            if (rl >= 0 && rl < a.M) {
                A.values(r, v);
                acc += A.gbar(r, -d, v);
            } else {
                // a boundary point of the neighbouring subdomain reads u^n_i
                // across its face; only an undelayed read lands on level n
                const long long pp = rl < 0 ? (p == 0 ? a.P - 1 : p - 1) : (p == a.P - 1 ? 0 : p + 1);
                const int ff = rl < 0 ? 1 : 0;
                if (A.delay(pp, ff) == 0) {
                    if (r < 0) r += a.N;
                    if (r >= a.N) r -= a.N;
                    A.values(r, v);
                    acc += A.gbar(r, -d, v);
                }
            }
        }
        // delayed reads from later steps addressed to level n
        if (loc < R) {
            T *q = A.pend(a.n, p, 0, (int)loc);
            acc += *q;
            *q = (T)0;
        } else if (loc >= a.M - R) {
            T *q = A.pend(a.n, p, 1, (int)(loc - (a.M - R)));
            acc += *q;
            *q = (T)0;
        }
        reinterpret_cast<T *>(a.lam_out)[i] = acc;

        // dJ/dnu: lambda^{n+1}_i (cB / nu) b_i
        A.values(i, v);
        T bv = (T)0;
#pragma unroll
        for (int q = -R; q <= R; ++q) bv += (T)Coeffs<ORDER>::beta(q) * v[q + R];
        nu_acc += (double)reinterpret_cast<const T *>(a.lam_in)[i] * a.dtdx2 * (double)bv;

        // this subdomain's delayed reads across a face, scattered to older
        // levels of the neighbour's boundary values (one thread per face)
        if (loc == 0 || loc == a.M - 1) {
            const int f = loc == 0 ? 0 : 1;
            const int k = A.delay(p, f);
            const long long q = f == 0 ? (p == 0 ? a.P - 1 : p - 1) : (p == a.P - 1 ? 0 : p + 1);
            T w[S_LEV];
            if constexpr (S_LEV == 2) {
                w[0] = (T)(k + 1);
                w[1] = (T)(-k);
            } else {
                w[0] = (T)((k + 1) * (k + 2) / 2);
                w[1] = (T)(-k * (k + 2));
                w[2] = (T)(k * (k + 1) / 2);
            }
            for (int t = 0; t < R; ++t) {
                const long long r = f == 0 ? i + t : i - t;           // reader point
                A.values(r, v);
                for (int j = (f == 0 ? -R : t + 1); j <= (f == 0 ? -t - 1 : R); ++j) {
                    const T gb = A.gbar(r, j, v);
                    // source: point (M + t + j) of q (face 0) or (j - t - 1) of q (face 1)
                    const int side = f == 0 ? 1 : 0;
                    const int sr = f == 0 ? R + t + j : j - t - 1;
                    for (int m = 0; m < S_LEV; ++m) {
                        if (k + m == 0 || w[m] == (T)0) continue;     // level n: gathered above
                        T *dst = A.pend(a.n - k - m, q, side, sr);
                        *dst += w[m] * gb;
                    }
                }
            }
        }
    }
    // per-block sum of the nu contributions, added to this block's running total
    __shared__ double red[256];
    red[threadIdx.x] = nu_acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.dnu_part[blockIdx.x] += red[0];
}

}  // namespace atk
