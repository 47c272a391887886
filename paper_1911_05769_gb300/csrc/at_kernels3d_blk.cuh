// at_kernels3d_blk.cuh -- temporally blocked free-running AT stepper for the
// scalar 3D Burgers equation (the equation and halos of at_kernels3d.cuh).
//
// A pass advances a subdomain by b levels (b <= L + 1, Sec. 3.2: a halo may
// be up to L levels old) with one read and one write of its state.  Level
// lv + i of a tile is updated plane by plane in a wavefront along z: at step
// t the CTA updates level lv + i at plane z = t - i + 1 for every i <= b, so
// level lv + i finds the three planes of level lv + i - 1 it needs one step
// after they were made.  Level lv comes from TMA plane copies of the state;
// a thread keeps the planes z - 1, z of every level for its own group of 4
// consecutive columns in registers, and levels lv + 1 .. lv + b - 1 of the
// current plane go to two alternating shared-memory planes per level for the
// y neighbours of other threads (x neighbours: warp shuffles).  Level lv + b
// is written in place.  One CTA barrier per step.
//
// Halos: at a tile start the CTA reads, per face, the neighbour's newest
// published level s <= lv and the one before it, f0 = entry(s) and
// d = entry(s) - entry(s - 1), and extrapolates the face's halo of every
// level lv + j of the pass (j < b) with delay k0 + j, k0 = lv - s, as
// f0 + (k0 + j) d (Eq. AT1/AT2 for two levels, in Newton form) into shared
// memory; the plane loop then only loads them (by address select in y, a
// predicated load in x).  The free-running rule: wait only until the
// neighbour has published level lv - min(L - b + 1, lv - 1), so the largest
// delay of the pass, k0 + b - 1, stays within L, and the delays of the
// start-up rule (two levels n - k, n - k - 1 >= 0) are met.  The first pass
// from level 0 takes one level.
//
// Neighbours only ever read levels that end a pass (a flag is released as the
// level a pass ends at, and passes of all subdomains start at the same
// levels), so a pass writes ring entries for its last two levels only (and
// for the launch's last L + 2 levels, which a later call of another mode may
// read).  A level collects the face values it publishes in its own halo
// arrays, at the words it has just read, and the whole CTA copies them to
// the ring after the tile's last step.  Delays are recorded per (level,
// subdomain, face) as in the unblocked stepper and replay exactly in the
// oracle.
#pragma once

#include "at_kernels3d.cuh"

namespace atk {

constexpr int kThreads3b = 256;    // threads of a CTA: one group of 4 columns each (planes <= 1024 points)
constexpr int kMaxPass3 = 4;       // levels per pass of the blocked stepper (2 .. 4, one instance each)
constexpr int kMaxStages3b = 8;    // plane stages at most (their barriers' space is fixed)

// shared memory: mbarriers and fill counts (space for kMaxStages3b stages),
// delay counters, the halos of the pass (face f, level j: array f * sb + j of
// `face_words` words; x faces [z][y], y faces [z][x], z faces [y][x]; after
// level j + 1 has read them, the faces it publishes), two planes per inner
// level, plane stages
struct Smem3b {
    long long bar_off, hist_off, halo_off, halo_bytes, lvl_off, plane_bytes, stage_off, total;
};

__host__ __device__ inline Smem3b smem3b_layout(int m0, int m1, long long face_words, int word, int stages, int sb)
{
    Smem3b l;
    l.bar_off = 0;                                   // full[stages], then one int per stage
    l.hist_off = 16LL * kMaxStages3b;               // (fixed: the offsets below do not depend on stages)
    l.halo_off = round_up(l.hist_off + 4LL * (kMaxL + 1), 128);
    l.halo_bytes = round_up(face_words * word, 16);
    l.lvl_off = round_up(l.halo_off + 6LL * sb * l.halo_bytes, 128);
    l.plane_bytes = round_up((long long)m0 * m1 * word, 128);
    l.stage_off = l.lvl_off + 2LL * (sb > 1 ? sb - 1 : 0) * l.plane_bytes;
    l.total = l.stage_off + (long long)stages * l.plane_bytes;
    return l;
}

template <int V>
struct IntC {
    static constexpr int value = V;
};

// levels of the pass that starts at level lv (the launch ends at level lev_end)
__host__ __device__ inline long long pass_len3(long long lv, long long lev_end, int sb)
{
    if (lv == 0) return 1;
    const long long r = lev_end - lv;
    return r < sb ? r : sb;
}

// BM: levels of a full pass (p.sb == BM); ISO: equal spacing on the three
// axes (one coefficient pair: the six neighbours summed before scaling); MS:
// 0, or the subdomain edge MS of cubic MS^3 subdomains known at compile time
// (every shared-memory offset and plane index then folds into constants)
template <typename T, int BM, bool ISO, int MS = 0>
__global__ void __launch_bounds__(kThreads3b, sizeof(T) == 4 ? 2 : 1)
    at_stepper3d_blk(const Params3 p, const __grid_constant__ CUtensorMap tmap)
{
    constexpr int NT = kThreads3b, VW = 4;
    extern __shared__ __align__(128) unsigned char smem[];
    const int NS = p.stages;
    const int m0 = MS ? MS : p.m0, m1 = MS ? MS : p.m1, m2 = MS ? MS : p.m2;
    const Smem3b sl = smem3b_layout(m0, m1, MS ? (long long)MS * MS : p.face_words, (int)sizeof(T), NS, BM);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + sl.bar_off);
    int *s_fills = reinterpret_cast<int *>(bars + NS);
    unsigned *hist = reinterpret_cast<unsigned *>(smem + sl.hist_off);
    // (32-bit offsets into shared memory)
    const int o_halo = (int)sl.halo_off, hb = (int)sl.halo_bytes, o_lvl = (int)sl.lvl_off,
              pbytes = (int)sl.plane_bytes, o_stage = (int)sl.stage_off;
    const int fw = MS ? MS * MS : (int)p.face_words;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long lo = (long long)blockIdx.x * p.P / p.G, hi = (long long)(blockIdx.x + 1) * p.P / p.G;
    const long long S = hi - lo;
    const long long lev0 = *reinterpret_cast<const volatile long long *>(p.ctrl + kCtrlN0);
    const long long lev_end = lev0 + p.n_steps;
    const int PW = m0 * m1;
    const unsigned plane_bytes = (unsigned)(PW * (int)sizeof(T));
    // passes: one level from level 0, then passes of BM levels (the last one shorter)
    const long long n_pass = lev0 == 0 ? 1 + (p.n_steps - 1 + BM - 1) / BM : (p.n_steps + BM - 1) / BM;
    const long long n_tiles = n_pass * S;
    const long long Q = n_tiles * m2;                       // planes this CTA reads
    constexpr bool F32 = sizeof(T) == 4;
    const T cA0 = F32 ? (T)p.cA32[0] : (T)p.cA[0], cA1 = F32 ? (T)p.cA32[1] : (T)p.cA[1],
            cA2 = F32 ? (T)p.cA32[2] : (T)p.cA[2];
    const T cB0 = F32 ? (T)p.cBf32[0][0] : (T)p.cB[0], cB1 = F32 ? (T)p.cBf32[0][1] : (T)p.cB[1],
            cB2 = F32 ? (T)p.cBf32[0][2] : (T)p.cB[2];

    if (tid < NS) {
        mbar_init(&bars[tid], 1);
        s_fills[tid] = 0;
    }
    if (tid == 0) mbar_fence_init();
    for (int i = tid; i <= kMaxL; i += NT) hist[i] = 0u;
    __syncthreads();

    const long long plane_words = p.n0 * p.n1;
    const unsigned uP0 = (unsigned)p.P0, uP01 = (unsigned)(p.P0 * p.P1);
    auto tile_coords = [&](long long sub, int *x, int *y, int *z) {
        const unsigned us = (unsigned)sub, q2 = us / uP01, r = us - q2 * uP01, q1 = r / uP0, q0 = r - q1 * uP0;
        *x = (int)(q0 * m0); *y = (int)(q1 * m1); *z = (int)(q2 * m2);
    };
    // plane z0 of the subdomain at (x0, y0) into stage st (thread 0 only)
    auto issue_plane = [&](int st, int x0, int y0, int z0) {
        mbar_arrive_expect_tx(&bars[st], plane_bytes);
        tensor_load_4d(smem + o_stage + st * pbytes, &tmap, x0, y0, z0, 0, &bars[st]);
        ++s_fills[st];
    };
    auto stage_at = [&](int st) -> const T * { return reinterpret_cast<const T *>(smem + o_stage + st * pbytes); };
    // halo array of face f at level j of the pass
    auto halo_at = [&](int f, int j) -> T * { return reinterpret_cast<T *>(smem + o_halo + (f * BM + j) * hb); };
    // Planes are waited for in order: ws, wp are the stage and fill parity of
    // the next one.  Lane 0 waits (bounded) and the warp follows.
    int ws = 0;
    unsigned wp = 0;
    auto wait_next = [&]() -> bool {
        int good = 1;
        if (lane == 0 && !mbar_try_wait(&bars[ws], wp)) good = wait_stage3(p, &bars[ws], wp) ? 1 : 0;
        good = __shfl_sync(0xffffffffu, good, 0);
        __syncwarp();
        if (++ws == NS) { ws = 0; wp ^= 1u; }
        return good != 0;
    };

    int tx0, ty0, tz0, nx0, ny0, nz0;
    tile_coords(lo, &tx0, &ty0, &tz0);
    tile_coords(lo + 1 == hi ? lo : lo + 1, &nx0, &ny0, &nz0);

    // this thread's group of 4 columns (rows of m0 / 4 <= 32 groups lie in
    // one warp).  Threads beyond the plane (small planes) take the first
    // group's addresses for their loads and store nothing.
    const int GR = m0 / VW;
    const bool cv = tid < PW / VW;
    const int cx = cv ? (tid % GR) * VW : 0, cy = cv ? tid / GR : 0, c = cy * m0 + cx;
    const int coff = cy * (int)p.n0 + cx;
    const bool fx0 = cx == 0, fx1 = cx + VW == m0, fy0 = cy == 0, fy1 = cy == m1 - 1;

    // level j of the pass (j = 0: the state read; j < b): planes z - 1, z of
    // this thread's columns while level j + 1 is at plane z, plane z in slot
    // z & 1 and plane z - 1 in the other
    T W[BM][2][VW];
#pragma unroll
    for (int j = 0; j < BM; ++j)
#pragma unroll
        for (int e = 0; e < VW; ++e) W[j][0][e] = W[j][1][e] = (T)0;

    if (tid == 0)
        for (int k = 0; k < NS && k < Q; ++k) issue_plane(k, tx0, ty0, tz0 + k);

    bool ok = true;
    long long lv = lev0, sub = lo;
    int b = (int)pass_len3(lv, lev_end, BM);
    long long prev_sub = -1, prev_new = 0;
    for (long long tt = 0; tt < n_tiles; ++tt) {
        const long long g0 = tt * m2;                        // this tile's first plane
        // ---- tile start: release the previous tile's flags, delays, halos
        __syncthreads();
        if (tid == 0 && prev_sub >= 0 && !(p.skip_publish && blockIdx.x == 0 && prev_new > p.skip_step)) {
            __threadfence();
            for (int f = 0; f < 6; ++f) st_release(p.flag + prev_sub * 6 + f, (unsigned long long)prev_new);
        }
        // one subdomain per CTA: the planes of this tile are the last tile's
        // output (fenced for the async proxy before the barrier above), read now
        if (tid == 0 && S == 1 && tt > 0) {
            int st = ws;
            for (int k = 0; k < NS && g0 + k < Q; ++k) {
                issue_plane(st, tx0, ty0, tz0 + k);
                if (++st == NS) st = 0;
            }
        }
        const unsigned us = (unsigned)sub, us2 = us / uP01, usr = us - us2 * uP01, us1 = usr / uP0;
        const long long s0 = usr - us1 * uP0, s1 = us1, s2 = us2;
        int bad = 0;
        if (warp < 6) {
            const int f = warp;
            const long long q = face_neighbour(p, s0, s1, s2, f);
            long long k0 = 0;
            int good = 1;
            if (lane == 0) {
                long long k0max = lv == 0 ? 0 : (long long)(p.L - b + 1);
                if (lv > 0 && k0max > lv - 1) k0max = lv - 1;
                const unsigned long long *fl = p.flag + q * 6 + (f ^ 1);
                unsigned long long seen = ld_acquire(fl);
                if ((long long)seen < lv - k0max && !wait_flag3(p, fl, lv - k0max, &seen, lv, q)) good = 0;
                if (good) {
                    k0 = lv - ((long long)seen < lv ? (long long)seen : lv);
                    for (int j = 0; j < b; ++j) {
                        atomicAdd(&hist[k0 + j], 1u);
                        if (p.delays) p.delays[((size_t)(lv + j - lev0) * p.P + sub) * 6 + f] = (int8_t)(k0 + j);
                    }
                } else {
                    atomicExch(p.ctrl + kCtrlAbort, 1);
                }
            }
            good = __shfl_sync(0xffffffffu, good, 0);
            k0 = __shfl_sync(0xffffffffu, k0, 0);
            if (good) {
                const T *e0 = ring_entry<T>(p, lv - k0, q, f ^ 1);
                // the older level is needed only if some level of the pass has a delay
                const bool dif = k0 + b - 1 > 0;
                const T *e1 = ring_entry<T>(p, lv - k0 - 1, q, f ^ 1);
                const int nw = f < 2 ? m1 * m2 : f < 4 ? m0 * m2 : m0 * m1;
                if ((nw & 3) == 0) {
                    // (several rows in flight: the tile start waits for these loads)
#pragma unroll 4
                    for (int i = 4 * lane; i < nw; i += 128) {
                        T v0[4], v1[4];
                        lds<T, 4>(e0 + i, v0);               // (a 16-byte generic load of global memory)
                        if (dif) lds<T, 4>(e1 + i, v1);
#pragma unroll
                        for (int e = 0; e < 4; ++e) v1[e] = dif ? v0[e] - v1[e] : (T)0;
#pragma unroll
                        for (int j = 0; j < BM; ++j) {
                            if (j >= b) break;
                            const T kk = (T)(k0 + j);
                            T h[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) h[e] = v0[e] + kk * v1[e];
                            sts4<T>(halo_at(f, j) + i, h);
                        }
                    }
                } else {
                    for (int i = lane; i < nw; i += 32) {
                        const T a = e0[i], d = dif ? a - e1[i] : (T)0;
                        for (int j = 0; j < b; ++j) halo_at(f, j)[i] = a + (T)(k0 + j) * d;
                    }
                }
            } else {
                bad = 1;
            }
        }
        if (__syncthreads_or(bad)) { ok = false; break; }
        T *uz = reinterpret_cast<T *>(p.u) + (((long long)tz0 * plane_words + (long long)ty0 * p.n0) + tx0) + coff;
        // the pass's last two levels go to the ring; levels from `ring_from`
        // on are published too (a later call of any mode may read the
        // launch's last L + 2 levels)
        const long long rf64 = lev_end - p.L - 1 - lv;
        const int ring_from = rf64 < 1 ? 1 : rf64 > BM + 1 ? BM + 1 : (int)rf64;
        // plane 0 of level lv
        int sc = ws;                                         // stage of plane t
        bad = wait_next() ? 0 : 1;
        if (!bad) lds<T, VW>(stage_at(sc) + c, W[0][0]);

        // level i (1 .. BM) of the pass at plane z = t - i + 1.  STEADY 1 / 2:
        // a step of the steady state (every level of a full pass at an
        // interior plane: no guards, no z faces) with t even / odd, so that
        // the window slots are known at compile time; 0: any step
        auto level = [&](auto I, auto STEADY, int t, int sn, T *up, const T *xh) {
            constexpr int i = decltype(I)::value, j = i - 1;
            constexpr bool ST = decltype(STEADY)::value != 0;
            constexpr int ZP = ((decltype(STEADY)::value - 1 - i + 1) % 2 + 2) % 2;   // z & 1 (steady)
            const int z = t - i + 1;
            if (!ST && (i > b || z < 0 || z >= m2)) return;   // (uniform over the CTA)
            const bool top = !ST && z == m2 - 1, bot = !ST && z == 0;
            // level j at plane z: the stage (j = 0) or the level's plane buffer
            const T *pl = j == 0 ? stage_at(sc)
                                 : reinterpret_cast<const T *>(smem + o_lvl + (2 * (j > 0 ? j - 1 : 0) + (z & 1)) * pbytes);
            T ab[VW], bl[VW], ym[VW], yp[VW], un[VW];
            if (top) lds<T, VW>(halo_at(5, j) + c, ab);
            else if (j == 0) lds<T, VW>(stage_at(sn) + c, ab);
            else {
#pragma unroll
                for (int e = 0; e < VW; ++e) ab[e] = up[e];
            }
            // level j at planes z (cw) and z - 1 from the window
            const bool odd = ST ? ZP != 0 : (z & 1) != 0;
            T cw[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                cw[e] = odd ? W[j][1][e] : W[j][0][e];
                bl[e] = odd ? W[j][0][e] : W[j][1][e];
            }
            if (bot) lds<T, VW>(halo_at(4, j) + c, bl);
            lds<T, VW>(fy0 ? halo_at(2, j) + z * m0 + cx : pl + c - m0, ym);
            lds<T, VW>(fy1 ? halo_at(3, j) + z * m0 + cx : pl + c + m0, yp);
            // x neighbours beyond the group: the neighbouring lanes' words,
            // or the x halos at a row's ends
            T xl = __shfl_up_sync(0xffffffffu, cw[VW - 1], 1);
            T xr = __shfl_down_sync(0xffffffffu, cw[0], 1);
            if (fx0) xl = xh[2 * j];
            if (fx1) xr = xh[2 * j + 1];
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const T cc = cw[e];
                const T xm = e == 0 ? xl : cw[e > 0 ? e - 1 : 0];
                const T xp = e == VW - 1 ? xr : cw[e + 1 < VW ? e + 1 : e];
                if constexpr (ISO) {
                    const T sum = ((xp + xm) + (yp[e] + ym[e])) + (ab[e] + bl[e]);
                    const T dif = ((xp - xm) + (yp[e] - ym[e])) + (ab[e] - bl[e]);
                    const T d2 = cB0 * (sum - (T)6 * cc);
                    un[e] = cc + (d2 - cc * (cA0 * dif));
                } else {
                    const T d2 = cB0 * ((xp + xm) - (T)2 * cc) + cB1 * ((yp[e] + ym[e]) - (T)2 * cc) +
                                 cB2 * ((ab[e] + bl[e]) - (T)2 * cc);
                    const T d1 = cA0 * (xp - xm) + cA1 * (yp[e] - ym[e]) + cA2 * (ab[e] - bl[e]);
                    un[e] = cc + (d2 - cc * d1);
                }
            }
            const bool last = ST ? i == BM : i == b;
            if (cv) {
                if (!last) sts4<T>(reinterpret_cast<T *>(smem + o_lvl + (2 * (i - 1) + (z & 1)) * pbytes) + c, un);
                else stv<T, VW>(uz + (long long)z * plane_words, un);
            }
            // the last two levels of the pass (and the launch's last L + 2)
            // go to the ring: their face values are kept in this level's
            // own halo arrays (level i read its halos of level lv + j at
            // these words above and reads them no more), and copied to the
            // ring by the whole CTA after the tile's last step
            const bool ring = ST ? (i + 1 >= BM || i >= ring_from) : (i + 1 >= b || i >= ring_from);
            if (ring && cv) {
                if (fx0) halo_at(0, j)[z * m1 + cy] = un[0];
                if (fx1) halo_at(1, j)[z * m1 + cy] = un[VW - 1];
                if (fy0) sts4<T>(halo_at(2, j) + z * m0 + cx, un);
                if (fy1) sts4<T>(halo_at(3, j) + z * m0 + cx, un);
                if (bot) sts4<T>(halo_at(4, j) + c, un);
                if (top) sts4<T>(halo_at(5, j) + c, un);
            }
            // level j's planes move up by one (plane z + 1 replaces plane
            // z - 1); level i starts its own window at plane 0; level i + 1
            // takes un as its plane above
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                if (odd) W[j][0][e] = ab[e];
                else W[j][1][e] = ab[e];
                if (i < BM && bot) W[i < BM ? i : 0][0][e] = un[e];
                up[e] = un[e];
            }
        };
        // one step of the wavefront: levels 1 .. BM, a CTA barrier (the
        // plane buffers written now are read at the next step; the stage of
        // plane t is free after it), the refill of that stage
        auto step = [&](int t, auto STEADY) -> bool {
            const int sn = ws;                               // stage of plane t + 1
            if (t + 1 < m2 && !bad) bad = wait_next() ? 0 : 1;
            if (!bad) {
                // the x halos of every level of the step, loaded first (their
                // latency then overlaps level 1 instead of each level's chain)
                T xh[2 * BM];
#pragma unroll
                for (int j = 0; j < BM; ++j) {
                    const int z = t - j;                     // plane of level j + 1
                    const bool act = decltype(STEADY)::value != 0 || (j < b && z >= 0 && z < m2);
                    xh[2 * j] = (act && fx0) ? halo_at(0, j)[z * m1 + cy] : (T)0;
                    xh[2 * j + 1] = (act && fx1) ? halo_at(1, j)[z * m1 + cy] : (T)0;
                }
                T up[VW];                                    // level i - 1 at plane z + 1 (this step)
                level(IntC<1>{}, STEADY, t, sn, up, xh);
                if constexpr (BM >= 2) level(IntC<2>{}, STEADY, t, sn, up, xh);
                if constexpr (BM >= 3) level(IntC<3>{}, STEADY, t, sn, up, xh);
                if constexpr (BM >= 4) level(IntC<4>{}, STEADY, t, sn, up, xh);
            }
            if (__syncthreads_or(bad)) return false;
            if (tid == 0 && t < m2) {
                const long long gq = g0 + t + NS;
                if (gq < Q) {
                    if (t + NS < m2) issue_plane(sc, tx0, ty0, tz0 + t + NS);
                    else if (S > 1) issue_plane(sc, nx0, ny0, nz0 + t + NS - m2);
                }
            }
            sc = sn;
            return true;
        };
        // ---- steps of the wavefront: a full pass runs its interior steps
        // (t = BM .. m2 - 2) in the steady form
        const int nst = m2 + b - 1;
        int t = 0;
        if (b == BM) {
            for (; t < BM && ok; ++t) ok = step(t, IntC<0>{});
            // (t = BM, BM + 1, ...: parities known at compile time)
            for (; t + 1 <= m2 - 2 && ok; t += 2) {
                ok = step(t, IntC<1 + (BM & 1)>{});
                if (ok) ok = step(t + 1, IntC<1 + ((BM + 1) & 1)>{});
            }
            if (t <= m2 - 2 && ok) ok = step(t++, IntC<1 + (BM & 1)>{});
        }
        for (; t < nst && ok; ++t) ok = step(t, IntC<0>{});
        if (!ok) break;
        // the faces of the levels published (in the halo arrays of the level
        // below them) to the ring: 16-byte copies spread over the CTA
        __syncthreads();
        {
            const int i_lo = (b - 1 < ring_from ? b - 1 : ring_from) < 1 ? 1 : (b - 1 < ring_from ? b - 1 : ring_from);
            for (int i = i_lo; i <= b; ++i) {
                T *rb = ring_entry<T>(p, lv + i, sub, 0);
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    const int nw = f < 2 ? m1 * m2 : f < 4 ? m0 * m2 : m0 * m1;
                    const T *h = halo_at(f, i - 1);
                    T *r = rb + (size_t)f * fw;
                    if ((nw & 3) == 0) {
                        for (int q = 4 * tid; q < nw; q += 4 * NT) {
                            T v[4];
                            lds<T, 4>(h + q, v);
                            stv<T, 4>(r + q, v);
                        }
                    } else {
                        for (int q = tid; q < nw; q += NT) r[q] = h[q];
                    }
                }
            }
        }
        // the next bulk read of this tile's output (its next pass) follows
        // a later barrier
        fence_proxy_async_global();
        prev_sub = sub;
        prev_new = lv + b;
        if (++sub == hi) {
            sub = lo;
            lv += b;
            b = (int)pass_len3(lv, lev_end, BM);
        }
        tx0 = nx0; ty0 = ny0; tz0 = nz0;
        tile_coords(sub + 1 == hi ? lo : sub + 1, &nx0, &ny0, &nz0);
    }
    __syncthreads();
    if (tid == 0 && ok && prev_sub >= 0 && !(p.skip_publish && blockIdx.x == 0 && prev_new > p.skip_step)) {
        __threadfence();
        for (int f = 0; f < 6; ++f) st_release(p.flag + prev_sub * 6 + f, (unsigned long long)prev_new);
    }
    // let the copies in flight land before leaving (bounded)
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

}  // namespace atk
