// at_kernels.cuh -- persistent weakly-synchronous AT stepper for sm_103a.
//
// One cooperative launch advances the whole 1D field by n_steps forward-Euler
// steps (arXiv 1911.05769, Sec. 3.2).  Every warp of the launch is one
// processing element (PE) of the paper: PE e owns the contiguous subdomains
// [lo, hi) and sweeps them in pass-major order.  A "tile" is one subdomain j
// over one pass of `len` consecutive levels n .. n+len (len = 1 except in
// blocked free-running mode).  For each tile the PE
//   * has already copied the subdomain's M state words into one of its
//     shared-memory stages with a bulk (TMA-engine) copy, D tiles ahead;
//   * has already chosen the delays k (prescribed, replayed, or -- free
//     running -- read off the neighbour's progress flag, blocking only while
//     the neighbour lags by more than the delay bound allows: the blocking
//     branch of Algorithm 2) and copied the neighbours' delayed boundary
//     values (levels n-k-m, Eq. AT1/AT2) from the ring buffers, one tile ahead;
//   * approximates the halo values ("approximate" step of Algorithm 2, split
//     form of Sec. 5.2), applies the unchanged central stencil of order 2 or
//     4 and the Euler update `len` times on the tile held in registers
//     (neighbour values by warp shuffles), and writes the final level back in
//     place;
//   * after every level writes the new boundary values into ring slot
//     (level mod T) and, on its two edge faces, releases the face's progress
//     flag (the notified put).
// Halo values never come from a neighbour's state array, only from the ring,
// so each PE updates its own subdomains in place, and a PE never waits for
// another PE of its CTA except through the same flags.
//
// Blocked free-running mode (temporal blocking): a pass of len <= L+1 levels
// uses, at inner step i, the halo extrapolated with delay k0 + i from the
// levels available when the pass started (Eq. AT1/AT2 with a larger k), so
// the state is read and written once per pass instead of once per level.
//
// AT_SYNC replaces the flag waits with a grid barrier between steps
// (Algorithm 1).  Every wait is bounded by timeout_ns; on expiry the kernel
// latches AT_ERR_TIMEOUT in the control block, raises the abort word and
// every PE leaves its loop (after its copies in flight have landed).
#pragma once

#include "at_device.cuh"

// Minimum resident CTAs per SM the stepper is compiled for (register cap).
#ifndef AT_MIN_CTAS_PER_SM
#define AT_MIN_CTAS_PER_SM 3
#endif
#ifndef AT_VGROUP
#define AT_VGROUP 2
#endif

namespace atk {

constexpr int kWarps = 4;                         // PEs (warps) per CTA
constexpr int kThreads = 32 * kWarps;
constexpr int kRingEntry = 16;                    // bytes per (slot, subdomain, face)
constexpr int kMaxS = 3;                          // levels per halo approximation
constexpr int kStripBytes = 64;                  // blocked synchronous mode: edge strip per (subdomain, face)
constexpr int kRawFace = 64;                      // raw bytes per face: kMaxS ring entries or one edge strip
constexpr int kRawBytes = 2 * kRawFace;           // one tile's delayed levels [face][m] (or edge strips)
constexpr int kMaxM = 1024;                       // points per subdomain (one warp's tile)
constexpr int kMaxL = 16;
constexpr int kMinStages = 2;                     // stages per PE (tile in use + one ahead)

enum : int { kModeSync = 0, kModeSeeded = 1, kModeFree = 2, kModeReplay = 3 };

// Shared-memory layout of one CTA, shared by the host (launch set-up) and the
// kernel: per PE `stages` mbarriers, delay counters, two raw-level buffers and
// `stages` tile buffers; then a table of `tab_bytes`: the forcing tables
// (sin/cos of the offsets in a subdomain, and of each PE's subdomain origins)
// or, for an ensemble, each PE's subdomain records.
struct SmemLayout {
    long long bar_off, hist_off, raw_off, stage_off, stage_bytes, tab_off, total;
};

__host__ __device__ inline long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }

// Groups of 4 points a lane of the stepper holds consecutively (see run_pe).
template <int GW, bool FULL, bool BATCH, int PREC>
__host__ __device__ constexpr int group_run() { return (!BATCH && FULL && PREC != 2 && GW % AT_VGROUP == 0) ? AT_VGROUP : 1; }

// Place of group g of a subdomain in the forcing tables: with runs of VG
// groups per lane the tables are stored run-slot-major, so that the lanes of
// a warp, reading slot i of their runs, read consecutive 16-byte words.
template <int VG>
__host__ __device__ inline int table_group(int g, int NG) { return VG == 1 ? g : (g % VG) * (NG / VG) + g / VG; }

__host__ __device__ inline SmemLayout smem_layout(long long M, int word, int stages, long long tab_bytes, bool comp = false)
{
    SmemLayout l;
    l.bar_off = 0;
    l.hist_off = round_up(8LL * kWarps * stages, 16);
    l.raw_off = round_up(l.hist_off + 4LL * kWarps * 2 * (kMaxL + 1), 128);
    l.stage_off = round_up(l.raw_off + 2LL * kWarps * kRawBytes, 128);
    l.stage_bytes = round_up(M * word, 128) * (comp ? 2 : 1);     // tile (+ its error words)
    l.tab_off = l.stage_off + (long long)kWarps * stages * l.stage_bytes;
    l.total = l.tab_off + tab_bytes;
    return l;
}

// Ensembles: independent 1D problems of M-point subdomains laid end to end.
// One record per subdomain (built on the host, copied to shared memory by the
// PE that owns it) and one per problem instance.
struct BatchSub {
    double cA, cB;             // stencil factors of the instance (as Params::cA, cB)
    unsigned long long seed;   // AT_SEEDED seed of the instance
    int L;                     // delay bound of the instance
    int lp;                    // index of the subdomain within its instance
    int Pi;                    // subdomains of the instance
    int inst;                  // instance
    long long left, right;     // global subdomain across face 0 / 1; -1 = exact boundary
    long long pad_;
};
static_assert(sizeof(BatchSub) == 64, "BatchSub is four 16-byte vectors");

struct BatchInst {
    double x0, dx, dt, nu;     // grid x_i = x0 + i dx of the instance, time step, viscosity
    double ta, tc, txc;        // exact boundary values u = c - a tanh(a (x - xc - c t) / (2 nu))
    double pad_;
};
static_assert(sizeof(BatchInst) == 64, "BatchInst is 64 bytes");

// A tile of an ensemble launch: cnt (1..ktile) consecutive subdomains s0 ..
// s0+cnt-1 of one instance, advanced together (the faces between them at
// delay 0: the neighbour's level itself).  Tiles are listed in the order the
// processing elements sweep them (instances grouped by delay bound); rec is
// the place of s0 in the list's enumeration of subdomains, which orders the
// subdomain records in shared memory.  link bit 0: the left neighbour of s0
// is the last subdomain of the previous tile of the list; bit 1: the right
// neighbour of the last subdomain is s0 of the next tile.  Stored as an int4
// (s0, rec, cnt | link << 16, 0).
struct TileInfo {
    long long s0, rec;
    int cnt, link;
};

struct Params {
    void *u;                   // state, N words, updated in place
    unsigned char *ring;       // [T][P][2] entries of 16 bytes
    unsigned long long *flag;  // [P][2] last level published per face
    int *ctrl;                 // control block (status, abort, diagnostics)
    unsigned long long *hist;  // [L+1] delay counts
    unsigned long long *gbar;  // grid-barrier arrival counter (AT_SYNC)
    int8_t *delays;            // [n_steps][P][2] replay input / record output
    const BatchSub *bsub;      // ensembles: [P] subdomain records (else NULL)
    const BatchInst *binst;    // ensembles: instance records (else NULL)
    const int4 *tiles;         // ensembles: the launch's tile list [ntiles] (see TileInfo)
    const int *sub_order;      // ensembles: subdomain at each place of the tile lists' enumeration [P]
    long long ntiles;          // tiles of the launch (single domain: P, tile j = subdomain j)
    int ktile;                 // most subdomains per tile
    void *ur;                  // compensated state: the rounding error of every point (N words)
    unsigned char *strip;      // blocked synchronous mode: edge strips [2][P][2] of kStripBytes (pass parity)
    int strip_words;           // words per strip (R x levels per pass, rounded up to a multiple of 4)
    void *levels;              // optional copy of every level l computed: slot l mod levels_depth of N words
    long long levels_depth;    // (single-level passes only; the adjoint's recomputation)
    long long N, P, M;
    int L, T, mode, per_sub;   // L: largest delay bound (ensembles: of any instance)
    long long n_steps;
    int sb;                    // most levels per pass (temporal blocking: free mode, and the blocked
                               // synchronous mode, where k = 0 and the ghost cells are recomputed)
    int alt;                   // sweep direction alternates from pass to pass (blocked free mode)
    unsigned long long seed;
    double cA, cB, dtA;        // dt/(2dx) | dt/(12dx);  nu dt/dx^2 | nu dt/(12dx^2);  dt A
    double x0, dx;
    int G;                     // CTAs
    int E;                     // PEs = G * kWarps
    int stages;                // tile buffers per PE
    long long smax;            // most subdomains of any PE
    long long bar_off, hist_off, raw_off, stage_off, stage_bytes, tab_off;
    long long timeout_ns;
    int skip_publish;          // test knob: PE 0 stops releasing flags
    long long skip_step;
};

// ---------------------------------------------------------------------------
// bounded waits
// ---------------------------------------------------------------------------
static __device__ __noinline__ void raise_timeout(const Params &p, int where, long long n, long long nb)
{
    if (atomicCAS(p.ctrl + kCtrlStatus, 0, kStatusTimeout) == 0) {
        p.ctrl[kCtrlCta] = (int)blockIdx.x;
        p.ctrl[kCtrlWhere] = where;
        p.ctrl[kCtrlNb] = (int)nb;
        p.ctrl[kCtrlStep] = (int)n;
    }
    atomicExch(p.ctrl + kCtrlAbort, 1);
}

// Waits until *fl >= need (acquire).  Returns the value seen in *seen.
static __device__ __noinline__ bool wait_flag(const Params &p, const unsigned long long *fl, long long need,
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

static __device__ __noinline__ bool wait_grid(const Params &p, unsigned long long target, long long n)
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
// quadratic through n-k, n-k-1, n-k-2.  k = 0 returns f^n itself.  Evaluated
// in Newton form, f0 + k d1 (+ k(k+1)/2 d2) with the backward differences
// d1 = f0 - f1, d2 = d1 - (f1 - f2): the same polynomial, but the
// differences of nearby levels are exact in floating point, so the rounding
// error stays about one ulp of f0 instead of growing with the weights
// (10, -15, 6 at k = 3).
template <typename T, int S_LEV>
__device__ __forceinline__ T approx_halo(const unsigned char *raw, int k, int r)
{
    const T r0 = reinterpret_cast<const T *>(raw)[r];
    if (k == 0) return r0;
    const T r1 = reinterpret_cast<const T *>(raw + kRingEntry)[r];
    const T d1 = r0 - r1;
    if constexpr (S_LEV == 2) {
        return r0 + (T)k * d1;
    } else {
        const T r2 = reinterpret_cast<const T *>(raw + 2 * kRingEntry)[r];
        const T d2 = d1 - (r1 - r2);
        return r0 + ((T)k * d1 + (T)(k * (k + 1) / 2) * d2);
    }
}

// Compensated state (PREC 2: a value is the pair hi + lo of FP32 words; ring
// entries hold the R hi words, then the R lo words): the halo value's hi word
// is the newest delayed level's hi word f0, and its lo word carries the rest
// of the same extrapolation in Newton form, f0 + k d1 (+ k(k+1)/2 d2 for
// s = 3), the backward differences d1, d2 formed word by word (differences of
// nearby hi words are exact), so that no part of the value is lost to the
// rounding of a single FP32 word.
template <typename T, int S_LEV, int R>
__device__ __forceinline__ T approx_halo_lo(const unsigned char *raw, int k, int r)
{
    const T *e0 = reinterpret_cast<const T *>(raw);
    const T h0 = e0[r], l0 = e0[R + r];
    if (k == 0) return l0;
    const T *e1 = reinterpret_cast<const T *>(raw + kRingEntry);
    const T h1 = e1[r], l1 = e1[R + r];
    const T d1 = (h0 - h1) + (l0 - l1);
    if constexpr (S_LEV == 2) {
        return l0 + (T)k * d1;
    } else {
        const T *e2 = reinterpret_cast<const T *>(raw + 2 * kRingEntry);
        const T h2 = e2[r], l2 = e2[R + r];
        const T d2 = ((h0 - h1) - (h1 - h2)) + ((l0 - l1) - (l1 - l2));
        return l0 + (T)k * d1 + (T)(k * (k + 1) / 2) * d2;
    }
}

// One 16-byte ring entry of a compensated FP32 state: R hi words, R lo words.
template <int R>
__device__ __forceinline__ void st_entry2(unsigned char *e, const float *h, const float *l)
{
    if constexpr (R == 2) st_cg16(e, h[0], h[1], l[0], l[1]);
    else st_cg16(e, h[0], l[0], 0.0f, 0.0f);
}

// One point of the forward-Euler update: w[0 .. 2R] are the values at offsets
// -R .. R (w[R] the point itself; wl the lo words of a compensated state),
// cA = dt/(2dx) | dt/(12dx), cB = nu dt/dx^2 | nu dt/(12dx^2) (cB64 the
// same in FP64), fs/fc and sv/cv the forcing factors of the subdomain and of
// the point's offset (A dt sin x = fs cv + fc sv); returns the new value
// (compensated state: updates the carried error too).  The stepper's tiles
// and the ghost cells of the blocked synchronous mode both call it, so a
// point computed twice is computed the same way twice.
template <typename T, int ORDER, bool FORCED, int PREC>
__device__ __forceinline__ T stencil_point(const T *w, const T *wl, T cA, T cB, double cB64, T fs, T fc, T sv, T cv,
                                           T &err)
{
    constexpr int R = ORDER / 2;
    const T cc = w[R];
    T a, b;
    if constexpr (PREC == 2) {
        // differences word by word; the second difference as differences
        // from the centre point
        const T cl = wl[R];
        if constexpr (ORDER == 2) {
            a = (w[2] - w[0]) + (wl[2] - wl[0]);
            b = ((w[2] - cc) + (w[0] - cc)) + ((wl[2] - cl) + (wl[0] - cl));
        } else {
            a = ((T)8 * (w[3] - w[1]) - (w[4] - w[0])) + ((T)8 * (wl[3] - wl[1]) - (wl[4] - wl[0]));
            b = ((T)16 * ((w[3] - cc) + (w[1] - cc)) - ((w[4] - cc) + (w[0] - cc))) +
                ((T)16 * ((wl[3] - cl) + (wl[1] - cl)) - ((wl[4] - cl) + (wl[0] - cl)));
        }
        T du = cB * b - cA * (cc + cl) * a;
        if constexpr (FORCED) du = fs * cv + (fc * sv + du);
        // two-sum of hi and (du + lo): exact sum t + err
        const T y = du + err;
        const T t = cc + y;
        const T yy = t - cc;
        err = (cc - (t - yy)) + (y - yy);
        return t;
    } else {
        (void)wl;
        (void)err;
        if constexpr (ORDER == 2) {
            a = w[2] - w[0];
            b = (w[2] + w[0]) - (T)2 * cc;
        } else {
            a = (T)8 * (w[3] - w[1]) - (w[4] - w[0]);
            b = (T)16 * (w[3] + w[1]) - (w[4] + w[0]) - (T)30 * cc;
        }
        if constexpr (PREC == 1) {
            double b64;
            if constexpr (ORDER == 2) {
                b64 = ((double)w[2] + (double)w[0]) - 2.0 * (double)cc;
            } else {
                b64 = 16.0 * ((double)w[3] + (double)w[1]) - ((double)w[4] + (double)w[0]) - 30.0 * (double)cc;
            }
            T rest = -cA * cc * a;
            if constexpr (FORCED) rest = fs * cv + (fc * sv + rest);
            (void)b;
            return (T)((double)cc + (cB64 * b64 + (double)rest));
        } else {
            (void)cB64;
            T du = cB * b - cA * cc * a;
            if constexpr (FORCED) du = fs * cv + (fc * sv + du);   // two fused multiply-adds
            return cc + du;
        }
    }
}

// Waits (lane 0) for the bulk copy into a stage; bounded.
static __device__ __noinline__ bool wait_stage(const Params &p, uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((long long)(global_ns() - t0) > p.timeout_ns) {
            raise_timeout(p, kWhereTile, -1, -1);
            return false;
        }
    }
}


// Synchronous algorithm: grid barrier before step `step` (1-based within the
// launch), combined per CTA.  Each warp counts itself on the CTA's shared
// counter; the warp completing the CTA's count arrives on the global counter
// and waits for all CTAs, then opens the CTA's epoch; the other warps wait
// for the epoch.  `wait` = false for the last arrival of a launch.  Bounded.
static __device__ __noinline__ bool cta_grid_sync(const Params &p, int *s_count, volatile long long *s_epoch,
                                                  long long step, bool wait)
{
    bool ok = true;
    if ((threadIdx.x & 31) == 0) {
        __threadfence();
        const int old = atomicAdd(s_count, 1);
        if ((long long)old + 1 == step * kWarps) {
            __threadfence();
            atomicAdd(p.gbar, 1ull);
            if (wait) ok = wait_grid(p, (unsigned long long)step * (unsigned long long)p.G, step);
            st_release_cta_shared(s_epoch, ok ? step : -1);
        } else if (wait) {
            const unsigned long long t0 = global_ns();
            long long ep;
            while ((ep = ld_acquire_cta_shared(s_epoch)) < step && ep >= 0) {
                if ((long long)(global_ns() - t0) > p.timeout_ns) { raise_timeout(p, kWhereGrid, step, -1); break; }
            }
            ok = (ep >= step);
        }
        __threadfence();
    }
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// The levels one launch advances a PE through: n0 .. n0 + n_steps, in passes
// of one level while the level is below s-1, then of sb levels (the last one
// shorter).  sb may differ between PEs (in an ensemble each PE takes the
// smallest delay bound of its subdomains): a PE's halo waits only need its
// neighbours' per-level flags, whatever their pass boundaries.
//
// alt: the sweep direction alternates from pass to pass (lo..hi-1, then
// hi-1..lo, ...).  A pass of L+1 levels must start from its edge neighbours'
// level n exactly (delay 0); in a one-way sweep the first tile of a pass
// needs the left neighbour PE's last tile of the previous pass, so every PE
// waits on its neighbour at each pass start.  Alternating, each edge tile
// needs a tile its neighbour finished about a pass earlier; and the tile at
// the turn is the same subdomain twice in a row, continued in registers.
//
// startup: passes of one level while the level is below s-1 (the AT halos
// need s levels); the synchronous modes read level n only and have none.
struct Sweep {
    long long n0, n_steps;
    int sb;
    bool alt;
    bool startup;
};

// Position of a tile in a PE's sweep: pass start level n, subdomain j, the
// pass length, (alternating sweeps) the direction of the pass, and the
// index of the pass within the launch.
struct Cursor {
    long long n, j;
    int len;
    bool rev;
    long long pass;
};

__device__ __forceinline__ int pass_len(const Sweep &sw, long long n, int s_lev)
{
    const long long left = sw.n0 + sw.n_steps - n;
    int len = (int)(left < sw.sb ? left : sw.sb);
    if (sw.startup && n < s_lev - 1) len = 1;
    return len;
}

__device__ __forceinline__ long long count_passes(const Sweep &sw, int s_lev)
{
    if (!sw.startup) return (sw.n_steps + sw.sb - 1) / sw.sb;
    long long single = (s_lev - 1) - sw.n0;
    if (single < 0) single = 0;
    if (single > sw.n_steps) single = sw.n_steps;
    const long long rest = sw.n_steps - single;
    return single + (rest + sw.sb - 1) / sw.sb;
}

__device__ __forceinline__ void advance(const Sweep &sw, Cursor &c, long long lo, long long hi, int s_lev)
{
    if (!sw.alt) {
        if (++c.j == hi) {
            c.j = lo;
            c.n += c.len;
            c.len = pass_len(sw, c.n, s_lev);
            ++c.pass;
        }
    } else if (c.rev ? c.j == lo : c.j == hi - 1) {
        // turn: the next pass starts on the same subdomain
        c.rev = !c.rev;
        c.n += c.len;
        c.len = pass_len(sw, c.n, s_lev);
        ++c.pass;
    } else {
        c.j += c.rev ? -1 : 1;
    }
}

// Exact boundary value of an ensemble instance (travelling tanh wave) at
// point `q` of the halo across face f of subdomain record b, at level lev.
template <int R>
static __device__ __noinline__ double exact_ghost64(const BatchInst *binst, const BatchSub &b, long long M, int f,
                                                    int q, long long lev)
{
    const BatchInst &bi = binst[b.inst];
    const long long gi = f ? ((long long)b.lp + 1) * M + q : (long long)b.lp * M - R + q;
    const double x = bi.x0 + (double)gi * bi.dx;
    const double t = (double)lev * bi.dt;
    return bi.tc - bi.ta * tanh(bi.ta * (x - bi.txc - bi.tc * t) / (2.0 * bi.nu));
}

template <typename T, int R>
__device__ __forceinline__ T exact_ghost(const BatchInst *binst, const BatchSub &b, long long M, int f, int q,
                                         long long lev)
{
    return (T)exact_ghost64<R>(binst, b, M, f, q, lev);
}

// The exact boundary value as a hi + lo pair of words (compensated state).
template <typename T, int R>
__device__ __forceinline__ T exact_ghost2(const BatchInst *binst, const BatchSub &b, long long M, int f, int q,
                                          long long lev, T &lo)
{
    const double g = exact_ghost64<R>(binst, b, M, f, q, lev);
    const T hi = (T)g;
    lo = (T)(g - (double)hi);
    return hi;
}

// ---------------------------------------------------------------------------
// one processing element (warp)
// ---------------------------------------------------------------------------
// Lane l keeps the 4-point groups g = l + 32 m (m < GW) of the tile in
// registers for the whole pass, so that loads and stores stay coalesced.  The
// left neighbours of group g are the last R words of group g-1 (lane l-1,
// same m; for lane 0, lane 31 at m-1), the right neighbours the first R words
// of group g+1 (lane l+1, same m; for lane 31, lane 0 at m+1): one shuffle
// per word, no barrier.  Groups 0 and NG-1 take the approximated halo instead.
//
// In an ensemble (BATCH) a tile is cnt consecutive subdomains of one instance
// (see TileInfo; the faces between them at delay 0); the stencil factors,
// delay bound and seed come from its records in shared memory; a face whose
// record names no neighbour takes the instance's exact boundary values,
// undelayed; a face whose neighbour is another PE's, or not in the adjacent
// tile of the sweep (a periodic instance's wrap-around), goes through the
// flags.
//
// PREC (FP32 state only) 1: the viscous term nu dt D2(u) is formed from the
// stencil values in FP64 and added to u in FP64, rounded to FP32 once per
// update (for runs close to the diffusive stability limit).  2: compensated
// state: every point is the pair hi + lo of FP32 words (lo: array p.ur, the
// rounding error of hi); the stencil differences are formed word by word
// (differences of nearby hi words are exact, those of the lo words small),
// the halo values and ring entries carry both words, and each update adds
// the increment and lo to hi with an error-free two-sum (Knuth), keeping the
// new error as lo -- so that neither small increments nor the quantisation
// of the stored field are lost to FP32 rounding.
template <typename T, int ORDER, int GW, bool FORCED, bool FULL, bool BATCH, int PREC, bool BS>
__device__ void run_pe(const Params &p, const Sweep &sw, long long lo, long long hi, uint64_t *bars, unsigned *hist,
                       unsigned char *raw, unsigned char *stages, const T *sj, const T *cj, const T *spt,
                       const T *cpt, const BatchSub *btab, int *s_count, volatile long long *s_epoch)
{
    constexpr int R = ORDER / 2;
    constexpr int S_LEV = ORDER / 2 + 1;
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long S = hi - lo;
    // Groups of 4 points a lane holds consecutively (full single-domain
    // tiles; else 1): register slot m of lane l is group
    // VG l + m mod VG + 32 VG (m div VG), so that a lane updates runs of VG
    // groups with register neighbours and exchanges words with its
    // neighbour lanes once per run instead of once per group.
    constexpr int VG = group_run<GW, FULL, BATCH, PREC>();
    auto gidx = [&](int m) -> int { return VG * lane + (m % VG) + 32 * VG * (m / VG); };
    // Blocked synchronous mode (AT_SYNC in passes of sb > 1 levels): every
    // delay is 0, a grid barrier precedes each pass, and a tile takes, instead
    // of the ring's per-level halo, its neighbours' edge strips of R sb points
    // at the pass's first level; the halo of each later level of the pass is
    // recomputed from them (ghost cells, the same arithmetic as the
    // neighbour's own update), so the result equals the unblocked AT_SYNC run
    // bit for bit.  Strips are written at the end of each pass (parity of the
    // pass index) and, at the launch start, from the state itself; barrier 1
    // follows that.
    // (a separate instantiation, BS: the host launches it for AT_SYNC with
    // passes of more than one level only)
    constexpr bool bsync = BS;
    const long long ep_off = bsync ? 1 : 0;                 // grid barriers before the first pass
    const long long n_ep = count_passes(sw, S_LEV) + ep_off; // arrivals of this launch
    if (S <= 0) {
        // a PE without subdomains still takes part in every grid barrier
        if (p.mode == kModeSync) {
            for (long long st = 1; st <= n_ep; ++st)
                if (!cta_grid_sync(p, s_count, s_epoch, st, st < n_ep)) break;
        }
        return;
    }
    // the subdomains of tile t (single domain: tile t is subdomain t)
    auto tile_info = [&](long long t) -> TileInfo {
        if constexpr (BATCH) {
            const int4 d = __ldg(p.tiles + t);
            return TileInfo{(long long)d.x, (long long)d.y, d.z & 0xffff, d.z >> 16};
        } else {
            return TileInfo{t, t, 1, 0};
        }
    };
    long long rec_lo = 0;                // place of this PE's first record
    if constexpr (BATCH) rec_lo = tile_info(lo).rec;
    // the first and last subdomain records of a tile (ensembles)
    auto rec_first = [&](const TileInfo &ti) -> const BatchSub & { return btab[ti.rec - rec_lo]; };
    auto rec_last = [&](const TileInfo &ti) -> const BatchSub & { return btab[ti.rec - rec_lo + ti.cnt - 1]; };
    // whether face f of tile t takes its halo through the flags: its
    // neighbour is not the adjacent tile of this PE's sweep (ensembles; the
    // single domain: the PE's first and last tile)
    auto link_edge = [&](long long t, const TileInfo &ti, int f) -> bool {
        return f == 0 ? !(t - 1 >= lo && (ti.link & 1)) : !(t + 1 < hi && (ti.link & 2));
    };
    const int NS = p.stages;
    // tiles loaded ahead; an alternating sweep revisits the subdomain of
    // position i after a turn 2i+1 tiles later, so at most 2 ahead there
    int D = (int)((S - 1) < (NS - 1) ? (S - 1) : (NS - 1));
    if (sw.alt && D > 2) D = 2;
    const long long Q = count_passes(sw, S_LEV) * S;
    // groups of 4 points in the tile (an ensemble's tiles: cnt subdomains)
    int NG = (int)(p.M / 4);
    // owner of group NG-1 (compile-time when the tile is a multiple of 128 points)
    int m_last = FULL ? GW - 1 : (NG - 1) >> 5;
    int lane_last = FULL ? 31 : (NG - 1) & 31;
    const T cA0 = (T)p.cA, cB0 = (T)p.cB;
    const double cB64_0 = p.cB;
    const size_t tile_bytes = (size_t)p.M * sizeof(T);                 // one subdomain
    const size_t slot_stride = (size_t)p.P * 2 * kRingEntry;
    const int up = (lane + 31) & 31, down = (lane + 1) & 31;
    const bool edge_pub = !(p.skip_publish && blockIdx.x == 0 && threadIdx.x < 32);
    unsigned *my_hist = hist + (lane & 1) * (kMaxL + 1);

    Cursor L{sw.n0, lo, pass_len(sw, sw.n0, S_LEV), false, 0};   // next tile to load
    Cursor H = L;                                     // next tile whose halo is prepared
    Cursor C = L;                                     // tile being processed

    // --- state tile copies (lane 0): tile t goes to stage t % NS ------------
    // (compensated state: the stage holds the tile, then its error words)
    const size_t err_off = round_up((long long)tile_bytes * p.ktile, 128);
    // (stage indices and phases are kept as running counters: no 64-bit
    // division per tile)
    auto issue_load = [&](int st, const Cursor &c) {
        if (lane == 0) {
            const TileInfo ti = tile_info(c.j);
            const size_t bytes = tile_bytes * (size_t)ti.cnt;
            uint64_t *bar = &bars[st];
            mbar_arrive_expect_tx(bar, (unsigned)(PREC == 2 ? 2 * bytes : bytes));
            bulk_load(stages + (size_t)st * p.stage_bytes,
                      reinterpret_cast<const unsigned char *>(p.u) + (size_t)ti.s0 * tile_bytes, (unsigned)bytes, bar);
            if constexpr (PREC == 2)
                bulk_load(stages + (size_t)st * p.stage_bytes + err_off,
                          reinterpret_cast<const unsigned char *>(p.ur) + (size_t)ti.s0 * tile_bytes, (unsigned)bytes,
                          bar);
        }
    };

    // --- halo preparation (lane f for face f) -------------------------------
    // Chooses the delay of face f of tile c and copies the delayed ring
    // levels into raw buffer `buf`.  With block == false an edge face whose
    // neighbour is not far enough yet is left pending (return 0); otherwise
    // waits (bounded).  Returns 1 when done, -1 on abort.
    int kb = 0;                        // lane i: raw delay of (tile t0 + i/2, face i%2)
    long long kb_t0 = -1;
    auto raw_delay = [&](long long t, const Cursor &c) -> int {
        // prescribed modes draw 16 tiles' delays at once (one per lane)
        const long long t0 = t & ~15LL;
        if (t0 != kb_t0) {
            // (n, j) of tile t0 + lane/2, stepping from c (tile t) back or forth
            long long jj = c.j - (t - t0) + (lane >> 1), nn = c.n;
            while (jj < lo) { jj += S; --nn; }
            while (jj >= hi) { jj -= S; ++nn; }
            int k = 0;
            if (t0 + (lane >> 1) < Q && nn >= sw.n0 && nn < sw.n0 + sw.n_steps) {
                // (prescribed delays: tiles of one subdomain)
                const TileInfo tj = tile_info(jj);
                if (p.mode == kModeSeeded) {
                    if constexpr (BATCH) {
                        const BatchSub &b = rec_first(tj);
                        k = seeded_delay(b.seed, nn, b.lp, b.Pi, p.per_sub ? 0 : (lane & 1), b.L);
                    } else {
                        k = seeded_delay(p.seed, nn, jj, p.P, p.per_sub ? 0 : (lane & 1), p.L);
                    }
                } else if (p.mode == kModeReplay) {
                    k = p.delays[((nn - sw.n0) * p.P + tj.s0) * 2 + (lane & 1)];
                }
            }
            kb = k;
            kb_t0 = t0;
        }
        const int i = 2 * (int)(t - t0);
        const int k0 = __shfl_sync(kAll, kb, i), k1 = __shfl_sync(kAll, kb, i + 1);
        return (lane & 1) ? k1 : k0;
    };

    int hk = 0;                        // lanes 0/1: delay at the start of the pass for the prepared tile
    auto prep_halo = [&](long long t, const Cursor &c, int buf, bool block) -> int {
        const int kr = (p.mode == kModeSeeded || p.mode == kModeReplay) ? raw_delay(t, c) : 0;
        // phase 1: choose the delay and check (or wait for) the neighbour
        int state = 1;
        long long k = 0, q = 0;
        bool bnd = false;              // exact boundary face (ensembles)
        const TileInfo ti = tile_info(c.j);
        if (lane < 2) {
            const int f = lane;
            const long long n = c.n;
            const int len = c.len;
            bool edge;
            int Lj = p.L;
            if constexpr (BATCH) {
                const BatchSub &bf = rec_first(ti), &bl = rec_last(ti);
                q = f ? bl.right : bf.left;
                bnd = q < 0;
                edge = !bnd && link_edge(c.j, ti, f);
                Lj = bf.L;
            } else {
                q = (f == 0) ? (c.j == 0 ? p.P - 1 : c.j - 1) : (c.j == p.P - 1 ? 0 : c.j + 1);
                edge = (f == 0) ? (c.j == lo) : (c.j == hi - 1);
            }
            // largest delay at the start of the pass such that the last inner
            // step stays within L, and no level below 0 is ever read
            long long kmax = n - S_LEV + 1;
            if (kmax < 0) kmax = 0;
            if (kmax > Lj - (len - 1)) kmax = Lj - (len - 1);
            k = kr;
            if (k > kmax) k = kmax;
            if (k < 0) k = 0;
            if (edge && p.mode != kModeSync) {
                const unsigned long long *fl = p.flag + q * 2 + (1 - f);
                const long long need = (p.mode == kModeFree) ? n - kmax : n - k;
                unsigned long long seen = ld_acquire(fl);
                if ((long long)seen < need) {
                    if (!block) state = 0;
                    else if (!wait_flag(p, fl, need, &seen, n, q)) state = -1;
                }
                if (state == 1 && p.mode == kModeFree) {
                    const long long avail = ((long long)seen < n) ? (long long)seen : n;
                    k = n - avail;
                }
            }
        }
        // the warp agrees: any lane aborted -> -1, else any lane pending -> 0
        const unsigned bad = __ballot_sync(kAll, state < 0), pend = __ballot_sync(kAll, state == 0);
        if (bad) return -1;
        if (pend) return 0;
        // phase 2: both faces ready -- count, record and copy the levels
        if (lane < 2) {
            const int f = lane;
            // (the synchronous modes use level n itself at every level: k = 0)
            const int kstep = p.mode == kModeSync ? 0 : 1;
            const long long sf = f ? ti.s0 + ti.cnt - 1 : ti.s0;      // the subdomain of face f
            for (int i = 0; i < c.len; ++i) {
                my_hist[k + kstep * i] += 1u;
                if (p.delays && p.mode != kModeReplay)
                    p.delays[((c.n - sw.n0 + i) * p.P + sf) * 2 + f] = (int8_t)(k + kstep * i);
            }
            if (BATCH && f == 0 && ti.cnt > 1) {
                // the faces between the tile's subdomains: delay 0
                for (int i = 0; i < c.len; ++i) {
                    my_hist[0] += 2u * (unsigned)(ti.cnt - 1);
                    if (p.delays && p.mode != kModeReplay)
                        for (int s = 0; s + 1 < ti.cnt; ++s) {
                            p.delays[((c.n - sw.n0 + i) * p.P + ti.s0 + s) * 2 + 1] = 0;
                            p.delays[((c.n - sw.n0 + i) * p.P + ti.s0 + s + 1) * 2 + 0] = 0;
                        }
                }
            }
            hk = (int)k;
            if constexpr (bsync) {
                // the neighbour's edge strip at the pass's first level
                const unsigned char *sb0 = p.strip +
                    ((size_t)((c.pass & 1) * p.P + (bnd ? 0 : q)) * 2 + (1 - f)) * kStripBytes;
                const int chunks = bnd ? 0 : p.strip_words * (int)sizeof(T) / 16;
                for (int ch = 0; ch < chunks; ++ch)
                    cp_async16(raw + (size_t)buf * kRawBytes + f * kRawFace + ch * 16, sb0 + ch * 16);
            } else {
                const unsigned char *rbase = p.ring + ((size_t)(bnd ? 0 : q) * 2 + (1 - f)) * kRingEntry;
                const int levels = bnd ? 0 : (k == 0 && c.len == 1) ? 1 : S_LEV;
                for (int m = 0; m < levels; ++m) {
                    const long long lv = c.n - k - m;
                    cp_async16(raw + (size_t)buf * kRawBytes + f * kRawFace + m * kRingEntry,
                               rbase + (size_t)(lv & (p.T - 1)) * slot_stride);
                }
            }
        }
        return 1;
    };

    // --- prologue -------------------------------------------------------------
    long long tl = 0;                  // next tile index to load
    long long nl = 0;                  // loads issued
    int sl = 0;                        // stage of the next load (nl % NS)
    int sr = 0;                        // stage of the next loaded tile to use and the parity of its fill
    unsigned ph = 0;
    // after a load: move to the next tile that is loaded (a turn tile of an
    // alternating sweep is not: it continues in registers)
    auto next_load = [&]() {
        const long long jj = L.j;
        advance(sw, L, lo, hi, S_LEV);
        ++tl;
        while (sw.alt && L.j == jj && tl < Q) { advance(sw, L, lo, hi, S_LEV); ++tl; }
        sl = (sl + 1 == NS) ? 0 : sl + 1;
        ++nl;
    };
    bool ok = true;
    if constexpr (bsync) {
        // edge strips of the state at the launch's first level (parity 0),
        // then the first grid barrier
        // (every subdomain of this PE's tiles: records rec_lo .. rec_hi-1)
        const int sw4 = p.strip_words;
        const T *ust = reinterpret_cast<const T *>(p.u);
        long long nrec = S;
        if constexpr (BATCH) {
            const TileInfo tl_ = tile_info(hi - 1);
            nrec = tl_.rec + tl_.cnt - rec_lo;
        }
        for (long long t = lane; t < nrec * 2 * sw4; t += 32) {
            const long long r = t / (2 * sw4);
            long long jj = lo + r;
            if constexpr (BATCH) jj = p.sub_order[rec_lo + r];
            const int f = (int)((t / sw4) & 1), wd = (int)(t % sw4);
            const long long src = jj * p.M + (f ? p.M - sw4 : 0) + wd;
            reinterpret_cast<T *>(p.strip + ((size_t)jj * 2 + f) * kStripBytes)[wd] = ust[src];
        }
        if (!cta_grid_sync(p, s_count, s_epoch, 1, true)) ok = false;
    }
    while (tl < D && tl < Q) { issue_load(sl, L); next_load(); }
    bool pending = true;               // the halo of tile 0 is prepared in the loop
    int k0cur = 0, k1cur = 0;
    bool turn = false;                 // tile r continues tile r-1 in registers (alternating sweep)
    T c[GW][4];                        // the tile's words, group g = lane + 32 m
    T er[PREC == 2 ? GW : 1][4];       // compensated state: carried rounding errors

    for (long long r = 0; r < Q && ok; ++r) {
        // state copy of tile r + D (stage of tile r - 1, complete: in order)
        if (tl < Q && tl <= r + D) { issue_load(sl, L); next_load(); }
        // synchronous algorithm: before the first tile of a pass (a step when
        // unblocked), all PEs have finished the previous pass (grid barrier,
        // Algorithm 1)
        if (p.mode == kModeSync && C.pass > 0 && C.j == lo) {
            if (!cta_grid_sync(p, s_count, s_epoch, C.pass + ep_off, true)) { ok = false; break; }
        }
        // halo of tile r: prepared one tile ahead unless it was pending
        const int buf = (int)(r & 1);
        if (pending) {
            if (prep_halo(r, C, buf, true) < 0) { ok = false; break; }
            H = C;
            advance(sw, H, lo, hi, S_LEV);
        }
        if (lane < 2) cp_async_wait_all();
        k0cur = __shfl_sync(kAll, hk, 0);
        k1cur = __shfl_sync(kAll, hk, 1);
        __syncwarp();
        // prepare the halo of tile r + 1 without blocking (in AT_SYNC it must
        // wait for the grid barrier when tile r + 1 starts a new step).  Its
        // internal right neighbour at the pass start was computed by tile
        // r + 2 - S, which is tile r itself when S == 2: no prefetch then.
        pending = true;
        if (r + 1 < Q && (S != 2 || sw.alt)) {
            const bool new_step = (H.j == lo);
            if (!(p.mode == kModeSync && new_step)) {
                const int st = prep_halo(r + 1, H, buf ^ 1, false);
                if (st < 0) { ok = false; break; }
                if (st > 0) {
                    pending = false;
                    advance(sw, H, lo, hi, S_LEV);
                }
            }
        }
        // the state tile (a turn tile is already in registers)
        const T *stile = reinterpret_cast<const T *>(stages + (size_t)sr * p.stage_bytes);
        if (!turn) {
            int good = 1;
            if (lane == 0 && !mbar_try_wait(&bars[sr], ph)) good = wait_stage(p, &bars[sr], ph);
            good = __shfl_sync(kAll, good, 0);
            __syncwarp();
            if (!good) { ok = false; break; }
            if (++sr == NS) { sr = 0; ph ^= 1u; }
        }
        const unsigned char *rw = raw + (size_t)buf * kRawBytes;
        const long long j = C.j, n = C.n;                 // tile, level at the pass start
        const int len = C.len;
        const TileInfo ti = tile_info(j);
        const long long s0 = ti.s0, s1 = ti.s0 + ti.cnt - 1;   // its first and last subdomain
        T *ug = reinterpret_cast<T *>(p.u) + (size_t)s0 * p.M;
        T cA = cA0, cB = cB0;
        double cB64 = cB64_0;
        bool bnd0 = false, bnd1 = false;
        if constexpr (BATCH) {
            const BatchSub &bf = rec_first(ti), &bl = rec_last(ti);
            cA = (T)bf.cA;
            cB = (T)bf.cB;
            cB64 = bf.cB;
            bnd0 = bf.left < 0;
            bnd1 = bl.right < 0;
            if constexpr (!FULL) {
                NG = (int)(ti.cnt * p.M / 4);
                m_last = (NG - 1) >> 5;
                lane_last = (NG - 1) & 31;
            }
        }

        if (!turn) {
#pragma unroll
            for (int m = 0; m < GW; ++m) {
                const int g = gidx(m);
                if (FULL || g < NG) lds<T, 4>(stile + 4 * g, c[m]);
                else { c[m][0] = c[m][1] = c[m][2] = c[m][3] = (T)0; }
                if constexpr (PREC == 2) {
                    const T *se =
                        reinterpret_cast<const T *>(reinterpret_cast<const unsigned char *>(stile) + err_off);
                    if (FULL || g < NG) lds<T, 4>(se + 4 * g, er[m]);
                    else { er[m][0] = er[m][1] = er[m][2] = er[m][3] = (T)0; }
                }
            }
        }
        // A sin(x) dt = (dt A sin x_j) cos(i dx) + (dt A cos x_j) sin(i dx)
        // (the tables hold subdomains lo-1 .. hi: entry j - lo + 1)
        T fs = (T)0, fc = (T)0;
        if constexpr (FORCED) {
            fs = (T)(p.dtA * (double)spt[j - lo + 1]);
            fc = (T)(p.dtA * (double)cpt[j - lo + 1]);
        }

        // blocked synchronous mode: ghost cells.  Lanes 0 .. G-1 hold the left
        // neighbour's points x = -G .. -1 (relative to the tile), lanes
        // 16 .. 16+G-1 the right neighbour's points M .. M+G-1, at the level
        // being advanced (G = R len; at the pass start, the strips)
        const int G = R * len;
        T gv = (T)0;
        T fsl = (T)0, fcl = (T)0, fsr = (T)0, fcr = (T)0;    // forcing factors of the neighbours
        if constexpr (bsync) {
            const T *stl = reinterpret_cast<const T *>(rw);
            const T *str = reinterpret_cast<const T *>(rw + kRawFace);
            if (lane < G) gv = stl[p.strip_words - G + lane];
            else if (lane >= 16 && lane < 16 + G) gv = str[lane - 16];
            if constexpr (FORCED) {
                fsl = (T)(p.dtA * (double)spt[j - lo]);
                fcl = (T)(p.dtA * (double)cpt[j - lo]);
                fsr = (T)(p.dtA * (double)spt[j - lo + 2]);
                fcr = (T)(p.dtA * (double)cpt[j - lo + 2]);
            }
        }

        // halo values of every inner level (delays k0 + i, k1 + i): lane
        // x < 2 R len computes one of them once per tile; each level then
        // takes its 2R values by shuffle
        const bool hv_lanes = !bsync && 2 * R * len <= 32;
        T hv = (T)0, hvl = (T)0;       // (hvl: lo word of a compensated state)
        if (hv_lanes && lane < 2 * R * len) {
            const int f = lane / (R * len), rem = lane % (R * len);
            const unsigned char *rf = rw + f * kRawFace;
            const int kf = (f ? k1cur : k0cur) + rem / R;
            if constexpr (PREC == 2) {
                if (BATCH && (f ? bnd1 : bnd0)) {
                    hv = exact_ghost2<T, R>(p.binst, f ? rec_last(ti) : rec_first(ti), p.M, f, rem % R, n + rem / R,
                                            hvl);
                } else {
                    hv = reinterpret_cast<const T *>(rf)[rem % R];
                    hvl = approx_halo_lo<T, S_LEV, R>(rf, kf, rem % R);
                }
            } else {
                if (BATCH && (f ? bnd1 : bnd0))
                    hv = exact_ghost<T, R>(p.binst, f ? rec_last(ti) : rec_first(ti), p.M, f, rem % R, n + rem / R);
                else
                    hv = approx_halo<T, S_LEV>(rf, kf, rem % R);
            }
        }
        // this lane's ring entry (slot 0) and flag of the face it publishes,
        // and whether the consumer across that face waits on the flag
        // (lane_last == 0: lane 0 publishes both faces, face 1 via prel1)
        const int pf = (lane == 0) ? 0 : 1;
        const long long sp = pf ? s1 : s0;                  // the subdomain of that face
        unsigned char *const pe0 = p.ring + ((size_t)sp * 2 + pf) * kRingEntry;
        unsigned long long *const pflag = p.flag + sp * 2 + pf;
        bool prel, prel1 = false;
        if constexpr (BATCH) {
            const BatchSub &bf = rec_first(ti), &bl = rec_last(ti);
            const long long q0 = pf ? bl.right : bf.left;
            prel = q0 >= 0 && link_edge(j, ti, pf);
            prel1 = bl.right >= 0 && link_edge(j, ti, 1);
        } else {
            prel = pf ? j == hi - 1 : j == lo;
            prel1 = j == hi - 1;
        }
        // one level of the tile, in place (cs and cd are the same array: a
        // group's old words are copied into its window before it is written)
        auto level = [&](int i, T (&cs)[GW][4], T (&cd)[GW][4]) {
            const long long lev = n + i + 1;                 // level being computed
            T hl[R], hr[R];
            T hll[R], hrl[R];                                // lo words (compensated state)
            if constexpr (bsync) {
                // the halo of level n+i from the ghost lanes (an ensemble's
                // domain ends: the exact values)
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    hll[q] = hrl[q] = (T)0;
                    hl[q] = __shfl_sync(kAll, gv, G - R + q);
                    hr[q] = __shfl_sync(kAll, gv, 16 + q);
                    if constexpr (BATCH) {
                        if (bnd0) hl[q] = exact_ghost<T, R>(p.binst, rec_first(ti), p.M, 0, q, n + i);
                        if (bnd1) hr[q] = exact_ghost<T, R>(p.binst, rec_last(ti), p.M, 1, q, n + i);
                    }
                }
                if (i + 1 < len) {
                    // the ghost cells of level n+i+1 from level n+i: ghost
                    // lanes and the tile's own edge words (not yet updated)
                    T el[R];
#pragma unroll
                    for (int q = 0; q < R; ++q) el[q] = (T)0;
#pragma unroll
                    for (int m = 0; m < GW; ++m) {
#pragma unroll
                        for (int q = 0; q < R; ++q) el[q] = (m == m_last) ? cs[m][4 - R + q] : el[q];
                    }
                    T ownl[R], ownr[R];
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        ownl[q] = __shfl_sync(kAll, cs[0][q], 0);
                        ownr[q] = __shfl_sync(kAll, el[q], lane_last);
                    }
                    const bool left = lane < 16;
                    const int xo = left ? lane - G : lane - 16;      // x, or x - M on the right
                    T w[2 * R + 1];
#pragma unroll
                    for (int jj = -R; jj <= R; ++jj) {
                        const T gq = __shfl_sync(kAll, gv, (lane + jj) & 31);
                        const int y = xo + jj;
                        T v;
                        if (left) v = (y < 0) ? gq : ((R == 1 || y == 0) ? ownl[0] : ownl[R - 1]);
                        else v = (y >= 0) ? gq : ((R == 1 || y == -1) ? ownr[R - 1] : ownr[0]);
                        w[jj + R] = v;
                    }
                    T sv = (T)0, cv = (T)0;
                    if constexpr (FORCED) {
                        if (left ? lane < G : lane - 16 < G) {
                            const int off = left ? (int)p.M + xo : xo;
                            const int tp = 4 * table_group<VG>(off >> 2, (int)(p.M / 4)) + (off & 3);
                            sv = sj[tp];
                            cv = cj[tp];
                        }
                    }
                    T unused = (T)0;
                    gv = stencil_point<T, ORDER, FORCED, PREC>(w, w, cA, cB, cB64, left ? fsl : fsr, left ? fcl : fcr,
                                                               sv, cv, unused);
                }
            } else {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                hll[q] = hrl[q] = (T)0;
                if (hv_lanes) {
                    hl[q] = __shfl_sync(kAll, hv, i * R + q);
                    hr[q] = __shfl_sync(kAll, hv, R * len + i * R + q);
                    if constexpr (PREC == 2) {
                        hll[q] = __shfl_sync(kAll, hvl, i * R + q);
                        hrl[q] = __shfl_sync(kAll, hvl, R * len + i * R + q);
                    }
                } else if constexpr (PREC == 2) {
                    const unsigned char *rr = rw + kRawFace;
                    if (BATCH && bnd0) {
                        hl[q] = exact_ghost2<T, R>(p.binst, rec_first(ti), p.M, 0, q, n + i, hll[q]);
                    } else {
                        hl[q] = reinterpret_cast<const T *>(rw)[q];
                        hll[q] = approx_halo_lo<T, S_LEV, R>(rw, k0cur + i, q);
                    }
                    if (BATCH && bnd1) {
                        hr[q] = exact_ghost2<T, R>(p.binst, rec_last(ti), p.M, 1, q, n + i, hrl[q]);
                    } else {
                        hr[q] = reinterpret_cast<const T *>(rr)[q];
                        hrl[q] = approx_halo_lo<T, S_LEV, R>(rr, k1cur + i, q);
                    }
                } else {
                    hl[q] = (BATCH && bnd0) ? exact_ghost<T, R>(p.binst, rec_first(ti), p.M, 0, q, n + i)
                                            : approx_halo<T, S_LEV>(rw, k0cur + i, q);
                    hr[q] = (BATCH && bnd1) ? exact_ghost<T, R>(p.binst, rec_last(ti), p.M, 1, q, n + i)
                                            : approx_halo<T, S_LEV>(rw + kRawFace, k1cur + i, q);
                }
            }
            }
            // One point: w[0 .. 2R] are the values at offsets -R .. R (w[R] the
            // point itself), sv/cv the forcing table entries; returns the new
            // value (compensated state: updates the carried error too).
            auto point = [&](const T *w, const T *wl, T sv, T cv, T &err) -> T {
                return stencil_point<T, ORDER, FORCED, PREC>(w, wl, cA, cB, cB64, fs, fc, sv, cv, err);
            };
            // lane l holds runs of VG groups of 4 points (group gidx(m) in
            // slot m); the neighbour words of a run come from the adjacent
            // lanes (lane 0 / 31: the other end of the warp at the previous /
            // next run, or the halo), those within a run from the lane's own
            // registers
            T tail[R], rb[R];                                // old last words of the previous run; new last words of NG-1
            T tail_l[R], rb_l[R];                            // (the same for the lo words, PREC 2)
#pragma unroll
            for (int q = 0; q < R; ++q) { tail[q] = (T)0; rb[q] = (T)0; tail_l[q] = (T)0; rb_l[q] = (T)0; }
#pragma unroll
            for (int b = 0; b < GW / VG; ++b) {
                const int mf = b * VG, ml = mf + VG - 1;     // the run's first and last slot
                T lh[R], rh[R];                              // words left of the run's first group, right of its last
                T lhl[R], rhl[R];
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const T to_next = (lane == 31) ? tail[q] : cs[ml][4 - R + q];
                    lh[q] = __shfl_sync(kAll, to_next, up);
                    const T to_prev = (lane == 0) ? cs[b + 1 < GW / VG ? mf + VG : mf][q] : cs[mf][q];
                    rh[q] = __shfl_sync(kAll, to_prev, down);
                    lhl[q] = rhl[q] = (T)0;
                    if constexpr (PREC == 2) {
                        const T ln = (lane == 31) ? tail_l[q] : er[ml][4 - R + q];
                        lhl[q] = __shfl_sync(kAll, ln, up);
                        const T lp = (lane == 0) ? er[b + 1 < GW / VG ? mf + VG : mf][q] : er[mf][q];
                        rhl[q] = __shfl_sync(kAll, lp, down);
                    }
                }
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    tail[q] = cs[ml][4 - R + q];
                    if constexpr (PREC == 2) tail_l[q] = er[ml][4 - R + q];
                }
                if (b == 0) {
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        lh[q] = (lane == 0) ? hl[q] : lh[q];
                        if constexpr (PREC == 2) lhl[q] = (lane == 0) ? hll[q] : lhl[q];
                    }
                }
                const bool is_last = (ml == m_last) && (lane == lane_last);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    rh[q] = is_last ? hr[q] : rh[q];
                    if constexpr (PREC == 2) rhl[q] = is_last ? hrl[q] : rhl[q];
                }
#pragma unroll
                for (int i = 0; i < VG; ++i) {
                    const int m = mf + i;
                    const int g = gidx(m);
                    T v[4 + 2 * R];
                    T vl[PREC == 2 ? 4 + 2 * R : 1];
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        v[q] = lh[q];
                        v[R + 4 + q] = (i == VG - 1) ? rh[q] : cs[m + 1 < GW ? m + 1 : m][q];
                        lh[q] = cs[m][4 - R + q];            // old words: the next group's left neighbours
                        if constexpr (PREC == 2) {
                            vl[q] = lhl[q];
                            vl[R + 4 + q] = (i == VG - 1) ? rhl[q] : er[m + 1 < GW ? m + 1 : m][q];
                            lhl[q] = er[m][4 - R + q];
                        }
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        v[R + e] = cs[m][e];
                        if constexpr (PREC == 2) vl[R + e] = er[m][e];
                    }
                    T s4[4], c4[4];
                    if constexpr (FORCED) {
                        // (full tiles: offsets known at compile time)
                        const int gg = (FULL || g < NG) ? g : NG - 1;
                        const int tg = table_group<VG>(gg, FULL ? 32 * GW : NG);
                        lds<T, 4>(sj + 4 * tg, s4);
                        lds<T, 4>(cj + 4 * tg, c4);
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        cd[m][e] = point(v + e, vl + (PREC == 2 ? e : 0), s4[e], c4[e],
                                         er[PREC == 2 ? m : 0][PREC == 2 ? e : 0]);
#pragma unroll
                    for (int q = 0; q < R; ++q) rb[q] = (m == m_last) ? cd[m][4 - R + q] : rb[q];
                    if constexpr (PREC == 2) {
#pragma unroll
                        for (int q = 0; q < R; ++q) rb_l[q] = (m == m_last) ? er[m][4 - R + q] : rb_l[q];
                    }
                }
            }
            // publish the new boundary values and release the edge flags
            // (face 0 by lane 0, face 1 by the owner of group NG-1; the
            // tile's entry addresses and release conditions are set above)
            if (lane == 0 || lane == lane_last) {
                const size_t slot_off = (size_t)(lev & (p.T - 1)) * slot_stride;
                const bool pub_ok = edge_pub || lev <= p.skip_step;
                if (FULL || lane_last != 0) {
                    T w[R], wl[R];             // word by word: no runtime choice between arrays
#pragma unroll
                    for (int q = 0; q < R; ++q) w[q] = pf ? rb[q] : cd[0][q];
                    if constexpr (PREC == 2) {
#pragma unroll
                        for (int q = 0; q < R; ++q) wl[q] = pf ? rb_l[q] : er[0][q];
                        st_entry2<R>(pe0 + slot_off, w, wl);
                    } else {
                        st_entry<T, R>(pe0 + slot_off, w);
                    }
                    if (p.mode == kModeSync) __threadfence();
                    if (prel && pub_ok) st_release(pflag, (unsigned long long)lev);
                } else {
                    // one group: lane 0 publishes both faces
#pragma unroll
                    for (int f = 0; f < 2; ++f) {
                        T w[R], wl[R];
#pragma unroll
                        for (int q = 0; q < R; ++q) w[q] = f ? rb[q] : cd[0][q];
                        if constexpr (PREC == 2) {
#pragma unroll
                            for (int q = 0; q < R; ++q) wl[q] = f ? rb_l[q] : er[0][q];
                            st_entry2<R>(pe0 + f * kRingEntry + slot_off, w, wl);
                        } else {
                            st_entry<T, R>(pe0 + f * kRingEntry + slot_off, w);
                        }
                        if (p.mode == kModeSync) __threadfence();
                        if ((f ? prel1 : prel) && pub_ok) st_release(pflag + f, (unsigned long long)lev);
                    }
                }
            }
            if constexpr (BATCH) {
                // the faces between the subdomains of a multi-subdomain tile
                // (subdomains of 128, 256 or 512 points: a subdomain's first
                // group is lane 0's, its last lane 31's): ring entries only,
                // and only of the launch's last L + s levels -- no tile of this
                // launch reads them, and a later launch with other tiles reads
                // back to its first level - L - s + 1 at most
                if (ti.cnt > 1 && (lane == 0 || lane == 31) && lev > sw.n0 + sw.n_steps - (p.L + S_LEV)) {
                    const size_t slot_off = (size_t)(lev & (p.T - 1)) * slot_stride;
                    const int gsh = p.M == 128 ? 0 : p.M == 256 ? 1 : 2;      // m slots per subdomain: 1 << gsh
                    const int gmask = (1 << gsh) - 1;
#pragma unroll
                    for (int m = 0; m < GW; ++m) {
                        const int sidx = m >> gsh;
                        const bool fst = lane == 0 && (m & gmask) == 0 && sidx >= 1 && sidx < ti.cnt;
                        const bool lst = lane == 31 && (m & gmask) == gmask && sidx + 1 < ti.cnt;
                        if (!(fst || lst)) continue;
                        const int fi = fst ? 0 : 1;
                        T w[R], wl[R];
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            w[q] = fst ? cd[m][q] : cd[m][4 - R + q];
                            wl[q] = (T)0;
                            if constexpr (PREC == 2) wl[q] = fst ? er[m][q] : er[m][4 - R + q];
                        }
                        unsigned char *e = p.ring + slot_off + ((size_t)(s0 + sidx) * 2 + fi) * kRingEntry;
                        if constexpr (PREC == 2) st_entry2<R>(e, w, wl);
                        else st_entry<T, R>(e, w);
                    }
                }
            }
        };
        for (int i = 0; i < len; ++i) level(i, c, c);
        if constexpr (bsync) {
            // edge strips of the pass's last level for the next pass
            const int gq = p.strip_words / 4;
            const size_t par_off = (size_t)((C.pass + 1) & 1) * p.P;
            T *st0 = reinterpret_cast<T *>(p.strip + ((par_off + s0) * 2 + 0) * kStripBytes);
            T *st1 = reinterpret_cast<T *>(p.strip + ((par_off + s1) * 2 + 1) * kStripBytes);
            // (read after the next grid barrier: the warp barrier at the end
            // of this tile and the fence of the arrival order them before it)
#pragma unroll
            for (int m = 0; m < GW; ++m) {
                const int g = gidx(m);
                if (g < gq) stg4<T>(st0 + 4 * g, c[m]);
                if (g >= NG - gq && g < NG) stg4<T>(st1 + 4 * (g - (NG - gq)), c[m]);
            }
        }
        // the next tile; before a turn the words stay in registers
        Cursor Cn = C;
        advance(sw, Cn, lo, hi, S_LEV);
        const bool keep = sw.alt && Cn.j == j && r + 1 < Q;
        if (!keep) {
#pragma unroll
            for (int m = 0; m < GW; ++m) {
                const int g = gidx(m);
                if (FULL || g < NG) stg4<T>(ug + 4 * g, c[m]);
                if constexpr (PREC == 2) {
                    if (FULL || g < NG) stg4<T>(reinterpret_cast<T *>(p.ur) + (size_t)s0 * p.M + 4 * g, er[m]);
                }
            }
        }
        if (p.levels) {
            T *lg = reinterpret_cast<T *>(p.levels) + (size_t)((n + len) % p.levels_depth) * (size_t)p.N +
                    (size_t)s0 * p.M;
#pragma unroll
            for (int m = 0; m < GW; ++m) {
                const int g = gidx(m);
                if (FULL || g < NG) stg4<T>(lg + 4 * g, c[m]);
            }
        }
        // the next read of this tile is a bulk copy (async proxy), issued by
        // lane 0 after the warp barrier
        fence_proxy_async_global();
        __syncwarp();
        C = Cn;
        turn = keep;
    }
    // synchronous algorithm: the last pass's arrival at the grid barrier
    if (ok && p.mode == kModeSync) cta_grid_sync(p, s_count, s_epoch, n_ep, false);
    // let every copy in flight land before the warp leaves
    if (lane < 2) cp_async_wait_all();
    if (lane == 0) {
        for (long long t = (nl > NS ? nl - NS : 0); t < nl; ++t) {
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(&bars[t % NS], (unsigned)((t / NS) & 1)) &&
                   (long long)(global_ns() - t0) < p.timeout_ns) {
            }
        }
    }
    __syncwarp();
    if (lane < 2) {
        for (int i = 0; i <= p.L && i <= kMaxL; ++i)
            if (my_hist[i]) atomicAdd(p.hist + i, (unsigned long long)my_hist[i]);
    }
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <typename T, int ORDER, int GW, bool FORCED, bool FULL, bool BATCH, int PREC, bool BS>
__global__ void __launch_bounds__(kThreads, AT_MIN_CTAS_PER_SM) at_stepper(const Params p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long e = (long long)blockIdx.x * kWarps + w;     // this warp's PE
    const long long lo = e * p.ntiles / p.E;                  // this PE's tiles
    const long long hi = (e + 1) * p.ntiles / p.E;
    const long long S = hi - lo;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + p.bar_off) + (size_t)w * p.stages;
    unsigned *hist = reinterpret_cast<unsigned *>(smem + p.hist_off) + (size_t)w * 2 * (kMaxL + 1);
    unsigned char *raw = smem + p.raw_off + (size_t)w * 2 * kRawBytes;
    unsigned char *stages = smem + p.stage_off + (size_t)w * p.stages * p.stage_bytes;
    T *tab = reinterpret_cast<T *>(smem + p.tab_off);
    T *sj = tab, *cj = tab + p.M;
    T *spt = tab + 2 * p.M + (size_t)w * 2 * (p.smax + 2), *cpt = spt + p.smax + 2;
    BatchSub *btab = reinterpret_cast<BatchSub *>(smem + p.tab_off) + (size_t)w * p.smax;
    // time level of the state, advanced at the end of the previous launch
    Sweep sw{*reinterpret_cast<const volatile long long *>(p.ctrl + kCtrlN0), p.n_steps, p.sb, p.alt != 0,
             p.mode != kModeSync};

    __shared__ int s_count;                   // grid-barrier arrivals of this CTA's warps
    __shared__ long long s_epoch;             // last grid barrier this CTA passed
    if (threadIdx.x == 0) { s_count = 0; s_epoch = 0; }
    if (lane == 0) {
        for (int i = 0; i < p.stages; ++i) mbar_init(&bars[i], 1);
        mbar_fence_init();
    }
    for (int i = lane; i < 2 * (kMaxL + 1); i += 32) hist[i] = 0u;
    if (FORCED) {
        // sin/cos of the offsets j dx within a subdomain and of the subdomain
        // origins x0 + p M dx (FP64), so that A sin(x_i) needs two FMAs
        for (long long i = threadIdx.x; i < p.M; i += blockDim.x) {
            double sv, cv;
            sincos((double)i * p.dx, &sv, &cv);
            constexpr int VG = group_run<GW, FULL, BATCH, PREC>();
            const long long tp = 4LL * table_group<VG>((int)(i >> 2), (int)(p.M / 4)) + (i & 3);
            sj[tp] = (T)sv;
            cj[tp] = (T)cv;
        }
        // entry i: subdomain lo - 1 + i (wrapped), i = 0 .. S + 1
        for (long long i = lane; i < S + 2; i += 32) {
            long long q = lo - 1 + i;
            if (q < 0) q += p.P;
            if (q >= p.P) q -= p.P;
            double sv, cv;
            sincos(p.x0 + (double)(q * p.M) * p.dx, &sv, &cv);
            spt[i] = (T)sv;
            cpt[i] = (T)cv;
        }
    }
    if constexpr (BATCH) {
        // this PE's subdomain records, in the order of its tiles; passes no
        // longer than the smallest delay bound among them allows
        // (k0 + len - 1 <= L), except in the synchronous modes
        long long r_lo = 0, r_hi = 0;
        if (S > 0) {
            const int4 a = p.tiles[lo], b = p.tiles[hi - 1];
            r_lo = a.y;
            r_hi = (long long)b.y + (b.z & 0xffff);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(btab);
        constexpr int kVec = (int)(sizeof(BatchSub) / sizeof(uint4));
        for (long long i = lane; i < (r_hi - r_lo) * kVec; i += 32)
            dst[i] = reinterpret_cast<const uint4 *>(p.bsub + p.sub_order[r_lo + i / kVec])[i % kVec];
        int lmin = kMaxL;
        for (long long i = lane; i < r_hi - r_lo; i += 32) lmin = min(lmin, p.bsub[p.sub_order[r_lo + i]].L);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
        if (p.mode != kModeSync && sw.sb > lmin + 1) sw.sb = lmin + 1;
    }
    __syncthreads();
    run_pe<T, ORDER, GW, FORCED, FULL, BATCH, PREC, BS>(p, sw, lo, hi, bars, hist, raw, stages, sj, cj, spt, cpt,
                                                       btab, &s_count, &s_epoch);
    // the last CTA to finish advances the level of the state and rearms the
    // grid barrier for the next launch (every CTA has read the level by now)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(p.ctrl + kCtrlDone, 1) == p.G - 1) {
            *reinterpret_cast<volatile long long *>(p.ctrl + kCtrlN0) = sw.n0 + p.n_steps;
            *reinterpret_cast<volatile int *>(p.ctrl + kCtrlDone) = 0;
            *reinterpret_cast<volatile unsigned long long *>(p.gbar) = 0ull;
            __threadfence();
        }
    }
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

// ---------------------------------------------------------------------------
// restart from stored levels: ring slots of levels lo_level .. level from the
// full fields levels[l mod depth], every flag at `level`, the control block
// cleared with the state's level set to `level`
// ---------------------------------------------------------------------------
template <typename T, int R>
__global__ void at_restore(const Params p, const T *levels, long long depth, long long lo_level, long long level)
{
    const long long nl = level - lo_level + 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const size_t slot_stride = (size_t)p.P * 2 * kRingEntry;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < p.P * nl; t += stride) {
        const long long j = t % p.P, l = lo_level + t / p.P;
        const T *u = levels + (size_t)(l % depth) * (size_t)p.N + (size_t)j * p.M;
        T a[2] = {u[0], R > 1 ? u[1] : (T)0};
        T b[2] = {u[p.M - R], R > 1 ? u[p.M - R + 1] : (T)0};
        unsigned char *e = p.ring + (size_t)(l & (p.T - 1)) * slot_stride + (size_t)j * 2 * kRingEntry;
        st_entry<T, R>(e, a);
        st_entry<T, R>(e + kRingEntry, b);
        if (l == level) {
            p.flag[j * 2 + 0] = (unsigned long long)level;
            p.flag[j * 2 + 1] = (unsigned long long)level;
        }
    }
    if (blockIdx.x == 0) {
        if (threadIdx.x < kCtrlWords) p.ctrl[threadIdx.x] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            *reinterpret_cast<long long *>(p.ctrl + kCtrlN0) = level;
            *p.gbar = 0ull;
        }
    }
}

}  // namespace atk

// ---------------------------------------------------------------------------
// kernel selection (each translation unit instantiates one word size and
// either the single-domain or the ensemble kernels)
// ---------------------------------------------------------------------------
namespace atk {

template <typename T, int ORDER, bool FORCED, bool FULL, bool BATCH, int PREC, bool BS>
void *stepper_gw(int gw)
{
    switch (gw) {
    case 1: return (void *)at_stepper<T, ORDER, 1, FORCED, FULL, BATCH, PREC, BS>;
    case 2: return (void *)at_stepper<T, ORDER, 2, FORCED, FULL, BATCH, PREC, BS>;
    case 4: return (void *)at_stepper<T, ORDER, 4, FORCED, FULL, BATCH, PREC, BS>;
    default: return (void *)at_stepper<T, ORDER, 8, FORCED, FULL, BATCH, PREC, BS>;
    }
}

template <typename T, int ORDER, bool FORCED, bool BATCH, int PREC, bool BS>
void *stepper_full(int gw, bool full)
{
    return full ? stepper_gw<T, ORDER, FORCED, true, BATCH, PREC, BS>(gw)
                : stepper_gw<T, ORDER, FORCED, false, BATCH, PREC, BS>(gw);
}

// Stepper for stencil order 2|4, gw groups of 4 points per lane (1, 2, 4 or
// 8), with or without forcing (single domain only), full tiles (M = 128 gw)
// or not; PREC 1: FP64 viscous accumulation, 2: compensated state; BS: the
// blocked synchronous mode (AT_SYNC in passes of more than one level).
template <typename T, bool BATCH, int PREC = 0, bool BS = false>
void *stepper_kernel(int order, int gw, bool forced, bool full)
{
    if constexpr (BATCH) {
        return order == 2 ? stepper_full<T, 2, false, true, PREC, BS>(gw, full)
                          : stepper_full<T, 4, false, true, PREC, BS>(gw, full);
    } else {
        if (order == 2)
            return forced ? stepper_full<T, 2, true, false, PREC, BS>(gw, full)
                          : stepper_full<T, 2, false, false, PREC, BS>(gw, full);
        return forced ? stepper_full<T, 4, true, false, PREC, BS>(gw, full)
                      : stepper_full<T, 4, false, false, PREC, BS>(gw, full);
    }
}

}  // namespace atk
