// at_api.cu -- host side of the C ABI declared in include/at.h.
//
// Validates arguments, carves the caller's workspace, chooses the launch shape
// of the persistent kernel (one CTA per SM, cooperative launch so that every
// CTA is resident and the bounded waits between CTAs always make progress),
// and launches the kernels on the caller's stream.  No device memory is
// allocated here.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include "at.h"
#include "at_adjoint.cuh"
#include "at_kernels.cuh"
#include "at_kernels3d_blk.cuh"

void *atk_stepper_kernel_f32(int order, int gw, bool forced, bool full);
void *atk_stepper_kernel_f32v(int order, int gw, bool forced, bool full);
void *atk_stepper_kernel_f32c(int order, int gw, bool forced, bool full);
void *atk_stepper_kernel_f64(int order, int gw, bool forced, bool full);
void *atk_sync_kernel_f32(int order, int gw, bool forced, bool full);
void *atk_sync_kernel_f32v(int order, int gw, bool forced, bool full);
void *atk_sync_kernel_f64(int order, int gw, bool forced, bool full);
void *atk_sync_batch_kernel_f32(int order, int gw, bool full);
void *atk_sync_batch_kernel_f64(int order, int gw, bool full);
void *atk_init_kernel_f32(int order);
void *atk_init_kernel_f64(int order);
void *atk_batch_kernel_f32(int order, int gw, bool full);
void *atk_batch_kernel_f64(int order, int gw, bool full);
void *atk_batch_kernel_f32c(int order, int gw, bool full);
void *atk_restore_kernel_f32(int order);
void *atk_restore_kernel_f64(int order);
void *atk_adjoint_kernel(int w, int order);
void *atk_adjoint_own_kernel(int w, int order);
void *atk_stepper3d_kernel(int w, int tc, int vw);
void *atk_stepper3d_iso_kernel(int w, int tc, int vw);
void *atk_system3d_kernel(int w, int tc, int nf, int vw);
void *atk_init3d_kernel(int w);
void *atk_stepper3d_blk_kernel(int w, int sb, int iso);
void *atk_stepper3d_blk32_kernel(int w, int sb, int iso);

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorCooperativeLaunchTooLarge)
        return fail(AT_ERR_RESIDENCY, "%s: %s", what, cudaGetErrorString(e));
    return fail(AT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int ring_slots(int L, int s)
{
    // A neighbour runs at most L+1 levels ahead of a consumer that reads back
    // to level n-L-s+1, so 2L+s+1 levels are live; round up to a power of 2.
    int need = 2 * L + s + 1, T = 1;
    while (T < need) T <<= 1;
    return T;
}

struct Layout {
    size_t u, ring, flag, ctrl, hist, gbar, bsub, binst, ur, strip, tiles, order, total;
};

// Workspace: state, ring buffers [T][P][2], flags [P][2], control block,
// delay counts, barrier counter; for an ensemble (n_inst > 0) also the
// subdomain and instance records.
Layout layout(int64_t N, int64_t P, int w, int L, int T, int64_t n_inst = 0, bool comp = false, bool strips = true)
{
    Layout l{};
    size_t off = 0;
    l.u = off;    off = align_up(off + (size_t)N * w, 256);
    l.ur = off;   // compensated state: the rounding error of every point
    if (comp) off = align_up(off + (size_t)N * w, 256);
    l.ring = off; off = align_up(off + (size_t)T * P * 2 * atk::kRingEntry, 256);
    l.flag = off; off = align_up(off + (size_t)P * 2 * 8, 256);
    l.ctrl = off; off = align_up(off + atk::kCtrlWords * 4, 256);
    l.hist = off; off = align_up(off + (size_t)(L + 1) * 8, 256);
    l.gbar = off; off = align_up(off + 8, 256);
    l.strip = off;   // blocked synchronous mode: edge strips [2][P][2]
    if (strips) off = align_up(off + (size_t)2 * P * 2 * atk::kStripBytes, 256);
    l.bsub = off; l.binst = off;
    l.tiles = off; l.order = off;
    if (n_inst > 0) {
        off = align_up(off + (size_t)P * sizeof(atk::BatchSub), 256);
        l.binst = off;
        off = align_up(off + (size_t)n_inst * sizeof(atk::BatchInst), 256);
        l.tiles = off;   // two tile lists [2][P] (one subdomain per tile; K per tile)
        off = align_up(off + (size_t)2 * P * sizeof(int4), 256);
        l.order = off;   // the lists' enumeration of the subdomains [P]
        off = align_up(off + (size_t)P * sizeof(int), 256);
    }
    l.total = off;
    return l;
}

// ---- three dimensions -------------------------------------------------------
struct Dims3 {
    int64_t n[3], P[3];
    int m[3];
    int64_t face_words;
};

int check_args3(const at_grid *g, int64_t P, int order, int L, Dims3 *d)
{
    if (g->bc != AT_BC_PERIODIC) return fail(AT_ERR_ARG, "bc must be AT_BC_PERIODIC");
    if (g->dtype != AT_F64 && g->dtype != AT_F32) return fail(AT_ERR_ARG, "dtype must be AT_F64 or AT_F32");
    if (order != 2) return fail(AT_ERR_ARG, "3D solvers use scheme_order 2");
    if (L < 0 || L > atk::kMaxL) return fail(AT_ERR_ARG, "L must be in 0..%d", atk::kMaxL);
    if (g->forcing_amp != 0.0) return fail(AT_ERR_ARG, "3D solvers are unforced");
    if (g->steps_per_pass < 0 || g->steps_per_pass > L + 1 || g->steps_per_pass > atk::kMaxPass3)
        return fail(AT_ERR_ARG, "3D steps_per_pass must be in 0..min(L+1, %d), got %d", atk::kMaxPass3,
                    g->steps_per_pass);
    int64_t np = 1;
    for (int a = 0; a < 3; ++a) {
        if (g->n[a] <= 0 || g->sub[a] <= 0 || g->n[a] % g->sub[a] != 0)
            return fail(AT_ERR_ARG, "axis %d: n=%lld is not a positive multiple of sub=%lld", a, (long long)g->n[a],
                        (long long)g->sub[a]);
        if (!(g->length[a] > 0.0)) return fail(AT_ERR_ARG, "length[%d] must be positive", a);
        d->n[a] = g->n[a];
        d->m[a] = (int)g->sub[a];
        d->P[a] = g->n[a] / g->sub[a];
        np *= d->P[a];
    }
    if (d->m[0] % 4 != 0) return fail(AT_ERR_ARG, "sub[0] must be a multiple of 4");
    if (d->m[0] > 256 || d->m[1] > 256) return fail(AT_ERR_ARG, "sub[0] and sub[1] must be <= 256");
    if ((int64_t)d->m[0] * d->m[1] > 1024) return fail(AT_ERR_ARG, "sub[0] * sub[1] must be <= 1024");
    if (d->m[1] < 2 || d->m[2] < 3) return fail(AT_ERR_ARG, "sub[1] >= 2 and sub[2] >= 3 are required");
    // blocked passes: a row of sub[0] / 4 groups of 4 columns lies within one warp
    if (g->steps_per_pass > 1 && (d->m[0] > 128 || (d->m[0] & (d->m[0] - 1)) != 0))
        return fail(AT_ERR_ARG, "3D steps_per_pass > 1 needs sub[0] a power of two in 4..128");
    if (P != np) return fail(AT_ERR_ARG, "P=%lld differs from the %lld subdomains of the grid", (long long)P, (long long)np);
    if (P >= (1LL << 31)) return fail(AT_ERR_ARG, "at most 2^31 - 1 subdomains (P=%lld)", (long long)P);
    int64_t fw = (int64_t)d->m[1] * d->m[2];
    if ((int64_t)d->m[0] * d->m[2] > fw) fw = (int64_t)d->m[0] * d->m[2];
    if ((int64_t)d->m[0] * d->m[1] > fw) fw = (int64_t)d->m[0] * d->m[1];
    d->face_words = (fw + 3) / 4 * 4;
    return AT_OK;
}

Layout layout3(const Dims3 &d, int64_t P, int w, int L, int T, int nf = 1)
{
    Layout l{};
    size_t off = 0;
    const int64_t N = d.n[0] * d.n[1] * d.n[2];
    l.u = off;    off = align_up(off + (size_t)nf * N * w, 256);
    l.ring = off; off = align_up(off + (size_t)T * P * 6 * nf * d.face_words * w, 256);
    l.flag = off; off = align_up(off + (size_t)P * 6 * 8, 256);
    l.ctrl = off; off = align_up(off + atk::kCtrlWords * 4, 256);
    l.hist = off; off = align_up(off + (size_t)(L + 1) * 8, 256);
    l.gbar = off; off = align_up(off + 8, 256);
    l.bsub = off; l.binst = off;   // (3D: per-block moment sums of at_moments, 4096 x 2 nf doubles)
    off = align_up(off + (size_t)4096 * 2 * nf * 8, 256);
    l.total = off;
    return l;
}

int check_args(const at_grid *g, int64_t P, int order, int L)
{
    if (!g) return fail(AT_ERR_ARG, "grid is NULL");
    if (g->dim == 3) {
        Dims3 d;
        return check_args3(g, P, order, L, &d);
    }
    if (g->dim != 1) return fail(AT_ERR_ARG, "dim must be 1 or 3");
    if (g->bc != AT_BC_PERIODIC) return fail(AT_ERR_ARG, "bc must be AT_BC_PERIODIC");
    if (g->dtype != AT_F64 && g->dtype != AT_F32) return fail(AT_ERR_ARG, "dtype must be AT_F64 or AT_F32");
    const int64_t N = g->n[0];
    if (N <= 0) return fail(AT_ERR_ARG, "n[0] must be positive");
    if (P <= 0 || N % P != 0) return fail(AT_ERR_ARG, "N %% P != 0 (N=%lld, P=%lld)", (long long)N, (long long)P);
    if (order != 2 && order != 4) return fail(AT_ERR_ARG, "scheme_order must be 2 or 4");
    if (L < 0 || L > atk::kMaxL) return fail(AT_ERR_ARG, "L must be in 0..%d", atk::kMaxL);
    const int64_t M = N / P;
    if (M % 4 != 0 || M < 4) return fail(AT_ERR_ARG, "M = N/P must be a multiple of 4 (M=%lld)", (long long)M);
    if (M > atk::kMaxM) return fail(AT_ERR_ARG, "M = N/P must be <= %d (M=%lld)", atk::kMaxM, (long long)M);
    if (!(g->length[0] > 0.0)) return fail(AT_ERR_ARG, "length[0] must be positive");
    if (g->steps_per_pass < 0 || g->steps_per_pass > L + 1)
        return fail(AT_ERR_ARG, "steps_per_pass must be in 0..L+1 (the delay bound), got %d", g->steps_per_pass);
    if (g->tile_subdomains > 1 || g->tile_subdomains < 0)
        return fail(AT_ERR_ARG, "tile_subdomains is for ensembles (0 or 1 for a single domain)");
    return AT_OK;
}

// Groups of 4 points each lane of a consumer warp keeps in registers: M/4
// groups over 32 lanes, rounded up to a power of two.
int groups_per_lane(int64_t M)
{
    const int64_t ng = M / 4;
    int g = 1;
    while ((int64_t)g * 32 < ng) g <<= 1;
    return g;
}

// Whether an FP32-state solver accumulates the viscous term in FP64: forced
// by the flags, else when nu dt / dx^2 reaches 0.8 of the stability limit.
bool viscous_fp64(int w, int order, uint32_t flags, double D)
{
    if (w != 4 || (flags & AT_FLAG_VISCOUS_FP32)) return false;
    if (flags & AT_FLAG_VISCOUS_FP64) return true;
    const double lim = order == 2 ? 0.5 : 0.375;
    return D >= 0.8 * lim;
}

// The stepper and init kernels for a word size, order, subdomain size,
// forcing and precision mode (instantiated in at_kernels_f32.cu,
// at_kernels_f32v.cu, at_kernels_f32c.cu and at_kernels_f64.cu).
void pick_kernels(int w, int order, int64_t M, bool forced, bool v64, bool comp, void **stepper, void **init,
                  void **stepper_bs = nullptr)
{
    const int gw = groups_per_lane(M);
    const bool full = (M == 128LL * gw);
    void *bs = nullptr;
    if (w == 8) {
        *stepper = atk_stepper_kernel_f64(order, gw, forced, full);
        bs = atk_sync_kernel_f64(order, gw, forced, full);
        *init = atk_init_kernel_f64(order);
    } else {
        *stepper = comp  ? atk_stepper_kernel_f32c(order, gw, forced, full)
                   : v64 ? atk_stepper_kernel_f32v(order, gw, forced, full)
                         : atk_stepper_kernel_f32(order, gw, forced, full);
        bs = comp ? nullptr : v64 ? atk_sync_kernel_f32v(order, gw, forced, full)
                                  : atk_sync_kernel_f32(order, gw, forced, full);
        *init = atk_init_kernel_f32(order);
    }
    if (stepper_bs) *stepper_bs = bs;
}

// Shared-memory table of a CTA: `fixed` bytes plus `per_sub` bytes per
// subdomain of each of its PEs and `extra` more subdomains per PE (forcing:
// sin/cos tables, which also cover the PE's two outer neighbours; ensembles:
// records); comp: stages hold the error words of a compensated state too.
struct TabSize {
    long long fixed, per_sub;
    bool comp;
    int extra;
    int64_t ntk;     // ensembles: tiles of the multi-subdomain list (0: single domain)
    int k;           // ensembles: most subdomains per tile
};

TabSize tab_size(int64_t M, int w, bool forced, bool batch, bool comp = false, int64_t ntk = 0, int k = 1)
{
    if (batch) return {0, (long long)sizeof(atk::BatchSub), comp, 0, ntk, k};
    if (forced) return {2LL * M * w, 2LL * w, comp, 2, 0, 1};
    return {0, 0, comp, 0, 0, 1};
}

// Chooses the CTA count (all co-resident CTAs unless max_ctas is set, at most
// one PE per subdomain) and the stages per PE that fit in shared memory, and
// sets the kernel's dynamic shared-memory size.
int launch_shape(int64_t M, int w, int64_t P, TabSize tsz, int max_ctas, int stages, int sms, int smem_optin,
                 void *kernel, int *G_out, int *stages_out, atk::SmemLayout *sl_out, int *smem_out,
                 long long *smax_out)
{
    if (M < 4 || M > atk::kMaxM) return fail(AT_ERR_ARG, "tile of %lld points (4..%d)", (long long)M, atk::kMaxM);
    auto layout_for = [&](int G, int st, long long *smax) {
        const int64_t E = (int64_t)G * atk::kWarps;
        // records per PE: the most tiles of one PE times the subdomains a tile
        // may have, over both tile lists of an ensemble
        *smax = (P + E - 1) / E;
        if (tsz.ntk > 0 && tsz.k > 1) {
            const long long sk = (tsz.ntk + E - 1) / E * tsz.k;
            if (sk > *smax) *smax = sk;
        }
        const long long tab = tsz.fixed + (long long)atk::kWarps * (*smax + tsz.extra) * tsz.per_sub;
        return atk::smem_layout(M, w, st, tab, tsz.comp);
    };
    // CTAs needed for one PE per subdomain at most
    const int gmax = (int)((P + atk::kWarps - 1) / atk::kWarps);
    int G = max_ctas > 0 ? max_ctas : sms;
    if (G > gmax) G = gmax;
    long long smax = 0;
    while (stages > atk::kMinStages && layout_for(G, stages, &smax).total > smem_optin) --stages;
    atk::SmemLayout sl = layout_for(G, stages, &smax);
    if (sl.total > smem_optin) return fail(AT_ERR_RESIDENCY, "shared memory %lld exceeds %d", sl.total, smem_optin);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl.total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, atk::kThreads, (size_t)sl.total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (max_ctas <= 0 && occ > 1) {
        // all co-resident CTAs (fewer subdomains per PE only shrinks the tables)
        int want = occ * sms;
        if (want > gmax) want = gmax;
        long long sm2 = 0;
        if (layout_for(want, stages, &sm2).total <= sl.total) { G = want; sl = layout_for(G, stages, &smax); }
    }
    if (occ < 1 || (int64_t)occ * sms < G)
        return fail(AT_ERR_RESIDENCY, "%d CTAs cannot be co-resident (occupancy %d per SM)", G, occ);
    *G_out = G;
    *stages_out = stages;
    *sl_out = sl;
    *smem_out = (int)sl.total;
    *smax_out = smax;
    return AT_OK;
}

}  // namespace

struct at_solver {
    at_grid g;
    int64_t N, P, M;
    int order, L, R, s, T, w;
    double nu, dt, dx;
    Layout lay;
    unsigned char *ws;
    cudaStream_t stream;
    int device, sm_count, smem_optin;
    int G, stages, sb, smem;
    long long smax;
    atk::SmemLayout sl;
    int64_t step;              // steps launched since at_set_state (host count)
    int64_t flags_E;           // PEs of the launch that last released flags (0: none since the state was set)
    bool has_state;
    int dim;                   // 1 or 3
    Dims3 d3;                  // 3D: extents, subdomains, ring entry size
    int tc;                    // 3D: columns per thread
    int nt3;                   // 3D: threads per CTA
    CUtensorMap tmap;          // 3D: tensor map of the state (planes of a subdomain, all fields)
    int nf;                    // 3D: fields (1: the scalar equation; 3..5: the system)
    double kappa[atk::kMaxFields3];   // 3D system: viscosity / diffusivities of the fields
    bool v64;                  // FP32 state with FP64 viscous accumulation
    bool comp;                 // FP32 state compensated by a second word per point
    bool batch;                // ensemble of instances
    int64_t n_inst;
    int lmin;                  // smallest delay bound (ensembles), else L
    int K;                     // ensembles: subdomains per tile of the AT_FREE / AT_SYNC list
    int64_t ntiles_k;          // ensembles: tiles of that list
    std::vector<atk::BatchSub> bsub_host;   // ensembles: the subdomain records (tile planning)
    std::vector<at_instance> inst_host;     // ensembles: the instances
    const void *flags_list;    // tile list of the launch that last released flags
    void *kernel;
    void *kernel_bs;           // the blocked synchronous mode's kernel (NULL: none)
    void *kernel_b3;           // 3D: the blocked free-running kernel (NULL: none)
    int G_b3, stages_b3, smem_b3;   // 3D: its CTAs, plane stages and shared memory
    bool bs_ok;                // it can run in the launch shape chosen for `kernel`
    void *init_kernel;
};

namespace {

// Sets every progress flag to the level of the state.  A launch releases
// only the flags of faces between processing elements; after a launch with
// another partition of the subdomains (another CTA count) the flags of faces
// that were inside a PE are stale, while every level up to the state's is
// complete and its ring entries are written (entries go out on every face).
__global__ void at_flags_to_level(unsigned long long *flag, const int *ctrl, long long nflags)
{
    const long long n0 = *reinterpret_cast<const long long *>(ctrl + atk::kCtrlN0);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nflags;
         i += (long long)gridDim.x * blockDim.x)
        flag[i] = (unsigned long long)n0;
}

// One launch of the persistent stepper: cooperative, so that every CTA is
// resident; cudaLaunchKernelExC with the cooperative attribute may be
// captured into a CUDA graph.  Brings the flags up to date first when the
// partition into PEs differs from the previous launch's.
cudaError_t launch_stepper(at_solver *h, atk::Params *p, void *kernel)
{
    const int64_t E = (int64_t)h->G * atk::kWarps;
    if (h->flags_E != 0 && (h->flags_E != E || h->flags_list != (const void *)p->tiles)) {
        const long long nflags = h->P * 2;
        const int blocks = (int)((nflags + 255) / 256 < 1024 ? (nflags + 255) / 256 : 1024);
        at_flags_to_level<<<blocks, 256, 0, h->stream>>>(p->flag, p->ctrl, nflags);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    h->flags_E = E;
    h->flags_list = p->tiles;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(h->G);
    cfg.blockDim = dim3(atk::kThreads);
    cfg.dynamicSmemBytes = (size_t)h->smem;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {p};
    return cudaLaunchKernelExC(&cfg, kernel, args);
}

// The blocked synchronous kernel runs in the launch shape chosen for the
// solver's kernel: the same dynamic shared memory, and only if as many of its
// CTAs can be resident (else AT_SYNC keeps one level per pass).
void prepare_bs(at_solver *h)
{
    h->bs_ok = false;
    if (!h->kernel_bs) return;
    if (cudaFuncSetAttribute(h->kernel_bs, cudaFuncAttributeMaxDynamicSharedMemorySize, h->smem) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, h->kernel_bs, atk::kThreads, (size_t)h->smem) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    h->bs_ok = (int64_t)occ * h->sm_count >= h->G;
}

// The tile lists of an ensemble.  Instances are taken in order of their
// delay bound (stable), so that the processing elements, which take
// contiguous runs of the lists, mostly hold instances of one bound and can
// make their passes L + 1 levels long; within an instance the subdomains are
// in order.  `order` enumerates the subdomains in that sequence; list 1 has
// one subdomain per tile, list K up to K consecutive subdomains of an
// instance per tile; both as atk::TileInfo int4s.
struct TilePlan {
    std::vector<int> order;
    std::vector<int4> list1, listk;
};

void plan_tiles(const std::vector<atk::BatchSub> &sub, int64_t n_inst, const at_instance *inst, int64_t M, int K,
                TilePlan *tp)
{
    std::vector<int64_t> first((size_t)n_inst);
    int64_t p0 = 0;
    for (int64_t j = 0; j < n_inst; ++j) { first[(size_t)j] = p0; p0 += inst[j].n / M; }
    std::vector<int64_t> idx((size_t)n_inst);
    for (int64_t j = 0; j < n_inst; ++j) idx[(size_t)j] = j;
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return inst[a].L < inst[b].L; });
    tp->order.clear();
    tp->list1.clear();
    tp->listk.clear();
    for (int64_t j : idx) {
        const int64_t Pi = inst[j].n / M, f0 = first[(size_t)j];
        const int64_t r0 = (int64_t)tp->order.size();
        for (int64_t lp = 0; lp < Pi; ++lp) {
            tp->order.push_back((int)(f0 + lp));
            tp->list1.push_back(make_int4((int)(f0 + lp), (int)(r0 + lp), 1, 0));
        }
        for (int64_t lp = 0; lp < Pi; lp += K) {
            const int cnt = (int)(Pi - lp < K ? Pi - lp : K);
            tp->listk.push_back(make_int4((int)(f0 + lp), (int)(r0 + lp), cnt, 0));
        }
    }
    // link bits: the neighbour across the tile's face is in the adjacent tile
    for (std::vector<int4> *l : {&tp->list1, &tp->listk}) {
        const int64_t n = (int64_t)l->size();
        for (int64_t t = 0; t < n; ++t) {
            int4 &d = (*l)[(size_t)t];
            const int cnt = d.z & 0xffff;
            int link = 0;
            if (t > 0) {
                const int4 &pv = (*l)[(size_t)(t - 1)];
                if (sub[(size_t)d.x].left == (long long)pv.x + (pv.z & 0xffff) - 1) link |= 1;
            }
            if (t + 1 < n && sub[(size_t)d.x + cnt - 1].right == (long long)(*l)[(size_t)(t + 1)].x) link |= 2;
            d.z = cnt | (link << 16);
        }
    }
}

// Ensembles: plans the tile lists for K subdomains per tile, copies them to
// the workspace (waits for the stream) and picks the kernels for tiles of up
// to K M points.
int set_tile_plan(at_solver *h, int K)
{
    TilePlan tp;
    plan_tiles(h->bsub_host, h->n_inst, h->inst_host.data(), h->M, K, &tp);
    unsigned char *tl = h->ws + h->lay.tiles;
    cudaError_t e = cudaMemcpyAsync(tl, tp.list1.data(), tp.list1.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                    h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tl + (size_t)h->P * sizeof(int4), tp.listk.data(), tp.listk.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->ws + h->lay.order, tp.order.data(), tp.order.size() * sizeof(int),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copying the tile lists");
    h->K = K;
    h->ntiles_k = (int64_t)tp.listk.size();
    const int gw = groups_per_lane((int64_t)K * h->M);
    const bool full = K == 1 && h->M == 128LL * gw;
    const int order = h->order;
    h->kernel = h->w == 8 ? atk_batch_kernel_f64(order, gw, full)
                : h->comp ? atk_batch_kernel_f32c(order, gw, full)
                          : atk_batch_kernel_f32(order, gw, full);
    h->kernel_bs = h->w == 8 ? atk_sync_batch_kernel_f64(order, gw, full)
                   : h->comp ? nullptr
                             : atk_sync_batch_kernel_f32(order, gw, full);
    h->flags_list = nullptr;
    return AT_OK;
}

}  // namespace

extern "C" {

const char *at_last_error(void) { return g_err; }

size_t at_workspace_bytes(const at_grid *grid, int64_t P, int scheme_order, int L)
{
    if (check_args(grid, P, scheme_order, L) != AT_OK) return 0;
    const int w = grid->dtype == AT_F64 ? 8 : 4;
    const int s = scheme_order / 2 + 1;
    if (grid->dim == 3) {
        Dims3 d;
        check_args3(grid, P, scheme_order, L, &d);
        return layout3(d, P, w, L, ring_slots(L, s), 1).total;
    }
    return layout(grid->n[0], P, w, L, ring_slots(L, s), 0, (grid->flags & AT_FLAG_COMPENSATED) != 0).total;
}

// nf = 1: the scalar equation with viscosity kappa[0]; nf = 3..5: the system
static int create3d(const at_grid *grid, int64_t P, int L, int nf, const double *kappa, double dt, at_solver **out)
{
    Dims3 d;
    int rc = check_args3(grid, P, 2, L, &d);
    if (rc != AT_OK) return rc;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(AT_ERR_ARG, "dt must be positive");
    double kmax = 0.0;
    for (int f = 0; f < nf; ++f) {
        if (!(kappa[f] >= 0.0) || !std::isfinite(kappa[f])) return fail(AT_ERR_ARG, "viscosity/diffusivity %d must be >= 0", f);
        if (kappa[f] > kmax) kmax = kappa[f];
    }
    double dx[3], sum = 0.0;
    for (int a = 0; a < 3; ++a) {
        dx[a] = grid->length[a] / (double)d.n[a];
        sum += 1.0 / (dx[a] * dx[a]);
    }
    if (!(grid->flags & AT_FLAG_ALLOW_UNSTABLE) && kmax * dt * sum > 0.5)
        return fail(AT_ERR_UNSTABLE, "kappa*dt*(1/dx^2+1/dy^2+1/dz^2) = %g exceeds 1/2", kmax * dt * sum);
    const int w = grid->dtype == AT_F64 ? 8 : 4;
    const int T = ring_slots(L, 2);
    const Layout lay = layout3(d, P, w, L, T, nf);
    if (!grid->workspace) return fail(AT_ERR_ARG, "workspace is NULL");
    if (grid->workspace_bytes < lay.total)
        return fail(AT_ERR_ARG, "workspace too small: %zu < %zu", grid->workspace_bytes, lay.total);
    if (reinterpret_cast<uintptr_t>(grid->workspace) % 256 != 0)
        return fail(AT_ERR_ARG, "workspace must be 256-byte aligned");
    int dev = 0, sms = 0, coop = 0, smem_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop) return fail(AT_ERR_RESIDENCY, "device does not support cooperative launch");

    // a thread takes one group of vw = 4 consecutive columns (FP32 planes of
    // 1024 points: every thread busy) or 1, 2 or 4 single columns
    const int pw = d.m[0] * d.m[1];
    // (a row of sub[0] / 4 groups must lie within one warp: sub[0] <= 128)
    const int vw = (w == 4 && d.m[0] % 4 == 0 && d.m[0] <= 128 && pw == 4 * atk::kThreads3) ? 4 : 1;
    // the scalar equation with groups of 4: CTAs of 128 threads, two groups
    // each (4 CTAs per SM: one CTA's tile start overlaps the others' planes)
    const int nt = (vw == 4 && nf == 1) ? 128 : atk::kThreads3;
    const int tc = vw == 4 ? (nf == 1 ? 2 : 1) : pw <= atk::kThreads3 ? 1 : pw <= 2 * atk::kThreads3 ? 2 : 4;
    if (nf > 1 && vw == 1 && tc > 2) return fail(AT_ERR_ARG, "the 3D system needs sub[0] * sub[1] <= 512 (or 1024, FP32)");
    const int sb = grid->steps_per_pass > 0 ? grid->steps_per_pass : 1;
    if (nf > 1 && sb > 1) return fail(AT_ERR_ARG, "the 3D system takes one level per pass");
    // (the scalar equation with equal spacing on the three axes: one
    // coefficient pair, the neighbours summed first)
    const int iso = dx[0] == dx[1] && dx[1] == dx[2];
    void *kern = nf == 1 ? (iso ? atk_stepper3d_iso_kernel(w, tc, vw) : atk_stepper3d_kernel(w, tc, vw))
                         : atk_system3d_kernel(w, tc, nf, vw);
    // plane buffers: at least 3 (planes z and z+1 in use, one arriving), at most sub[2]
    int stages = grid->stages > 0 ? grid->stages : 4;
    if (stages < 3) stages = 3;
    if (stages > d.m[2]) stages = d.m[2];
    atk::Smem3 sl3 = atk::smem3_layout(d.m[0], d.m[1], d.m[2], w, stages, nf);
    while (sl3.total > smem_optin && stages > 3) sl3 = atk::smem3_layout(d.m[0], d.m[1], d.m[2], w, --stages, nf);
    if (sl3.total > smem_optin) return fail(AT_ERR_RESIDENCY, "shared memory %lld exceeds %d", sl3.total, smem_optin);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl3.total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, (size_t)sl3.total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    int64_t G = grid->max_ctas > 0 ? grid->max_ctas : (int64_t)occ * sms;
    if (G > P) G = P;
    if (occ < 1 || (int64_t)occ * sms < G)
        return fail(AT_ERR_RESIDENCY, "%lld CTAs cannot be co-resident (occupancy %d per SM)", (long long)G, occ);

    at_solver *h = new (std::nothrow) at_solver();
    if (!h) return fail(AT_ERR_ARG, "out of host memory");
    h->g = *grid;
    if (h->g.timeout_ns <= 0) h->g.timeout_ns = 1000000000ll;
    h->dim = 3;
    h->d3 = d;
    h->tc = tc;
    h->nt3 = nt;
    h->nf = nf;
    for (int f = 0; f < nf; ++f) h->kappa[f] = kappa[f];
    h->N = (int64_t)nf * d.n[0] * d.n[1] * d.n[2];   // words of the state (all fields)
    h->P = P;
    h->M = (int64_t)d.m[0] * d.m[1] * d.m[2];
    h->order = 2; h->L = L; h->R = 1; h->s = 2; h->T = T; h->w = w;
    h->nu = kappa[0]; h->dt = dt; h->dx = dx[0];
    h->lay = lay;
    h->ws = static_cast<unsigned char *>(grid->workspace);
    h->stream = static_cast<cudaStream_t>(grid->stream);
    h->device = dev; h->sm_count = sms; h->smem_optin = smem_optin;
    h->kernel = kern;
    h->init_kernel = atk_init3d_kernel(w);
    h->G = (int)G;
    h->stages = stages;
    h->smem = (int)sl3.total;
    h->sb = sb;
    h->lmin = L;
    h->kernel_b3 = nullptr;
    if (sb > 1) {
        // the blocked free-running kernel: 256 threads (a group of 4 columns
        // each), its own plane stages (2 in use, the rest arriving) and grid
        // (32^3 subdomains: the instances with the sizes known at compile time)
        const bool cube32 = d.m[0] == 32 && d.m[1] == 32 && d.m[2] == 32;
        void *kb = cube32 ? atk_stepper3d_blk32_kernel(w, sb, iso) : atk_stepper3d_blk_kernel(w, sb, iso);
        int st = grid->stages > 0 ? grid->stages : 4;
        if (st < 3) st = 3;
        if (st > atk::kMaxStages3b) st = atk::kMaxStages3b;
        if (st > d.m[2]) st = d.m[2];
        atk::Smem3b sb3 = atk::smem3b_layout(d.m[0], d.m[1], d.face_words, w, st, sb);
        while (sb3.total > smem_optin && st > 3) sb3 = atk::smem3b_layout(d.m[0], d.m[1], d.face_words, w, --st, sb);
        if (sb3.total > smem_optin) {
            delete h;
            return fail(AT_ERR_RESIDENCY, "blocked 3D passes: shared memory %lld exceeds %d", sb3.total, smem_optin);
        }
        e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb3.total);
        if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaFuncSetAttribute"); }
        int occb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occb, kb, atk::kThreads3b, (size_t)sb3.total);
        if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor"); }
        int64_t Gb = grid->max_ctas > 0 ? grid->max_ctas : (int64_t)occb * sms;
        if (Gb > P) Gb = P;
        if (occb < 1 || (int64_t)occb * sms < Gb) {
            delete h;
            return fail(AT_ERR_RESIDENCY, "blocked 3D passes: %lld CTAs cannot be co-resident (occupancy %d per SM)",
                        (long long)Gb, occb);
        }
        h->kernel_b3 = kb;
        h->G_b3 = (int)Gb;
        h->stages_b3 = st;
        h->smem_b3 = (int)sb3.total;
    }
    // tensor map of the state: boxes of sub[0] x sub[1] x 1 points (one plane
    // of a subdomain), encoded through the driver entry point of the runtime
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    cudaDriverEntryPointQueryResult qres = cudaDriverEntryPointSymbolNotFound;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", reinterpret_cast<void **>(&encode), 12000,
                                         cudaEnableDefault, &qres);
    if (e != cudaSuccess || qres != cudaDriverEntryPointSuccess || !encode) {
        delete h;
        return fail(AT_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    }
    // 4D: x, y, z, field; a box is one plane of a subdomain in every field
    const cuuint64_t gdim[4] = {(cuuint64_t)d.n[0], (cuuint64_t)d.n[1], (cuuint64_t)d.n[2], (cuuint64_t)nf};
    const cuuint64_t gstride[3] = {(cuuint64_t)(d.n[0] * w), (cuuint64_t)(d.n[0] * d.n[1] * w),
                                   (cuuint64_t)(d.n[0] * d.n[1] * d.n[2] * w)};
    const cuuint32_t box[4] = {(cuuint32_t)d.m[0], (cuuint32_t)d.m[1], 1u, (cuuint32_t)nf};
    const cuuint32_t estride[4] = {1u, 1u, 1u, 1u};
    const CUresult cr = encode(&h->tmap, w == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                               h->ws + lay.u, gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        delete h;
        return fail(AT_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    }
    *out = h;
    return AT_OK;
}

static atk::Params3 make_params3(const at_solver *h)
{
    atk::Params3 p{};
    p.u = h->ws + h->lay.u;
    p.ring = h->ws + h->lay.ring;
    p.flag = reinterpret_cast<unsigned long long *>(h->ws + h->lay.flag);
    p.ctrl = reinterpret_cast<int *>(h->ws + h->lay.ctrl);
    p.hist = reinterpret_cast<unsigned long long *>(h->ws + h->lay.hist);
    p.gbar = reinterpret_cast<unsigned long long *>(h->ws + h->lay.gbar);
    p.n0 = h->d3.n[0]; p.n1 = h->d3.n[1]; p.n2 = h->d3.n[2];
    p.m0 = h->d3.m[0]; p.m1 = h->d3.m[1]; p.m2 = h->d3.m[2];
    p.P0 = h->d3.P[0]; p.P1 = h->d3.P[1]; p.P2 = h->d3.P[2]; p.P = h->P;
    p.L = h->L; p.T = h->T; p.stages = h->stages;
    p.seed = h->g.seed;
    for (int a = 0; a < 3; ++a) {
        const double dxa = h->g.length[a] / (double)h->d3.n[a];
        p.cA[a] = h->dt / (2.0 * dxa);
        p.cB[a] = h->nu * h->dt / (dxa * dxa);
        for (int f = 0; f < h->nf; ++f) p.cBf[f][a] = h->kappa[f] * h->dt / (dxa * dxa);
        p.cA32[a] = (float)p.cA[a];
        for (int f = 0; f < atk::kMaxFields3; ++f)
            p.cBf32[f][a] = (float)(h->nf > 1 ? (f < h->nf ? p.cBf[f][a] : 0.0) : p.cB[a]);
    }
    p.nf = h->nf;
    p.skip_publish = (h->g.flags & AT_FLAG_TEST_SKIP_PUBLISH) ? 1 : 0;
    p.skip_step = h->g.test_skip_step;
    p.face_words = h->d3.face_words;
    p.G = h->G;
    p.timeout_ns = h->g.timeout_ns;
    return p;
}

int at_create(const at_grid *grid, int64_t P, int scheme_order, int L, double nu, double dt, at_solver **out)
{
    g_err[0] = 0;
    if (!out) return fail(AT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (grid && grid->dim == 3) return create3d(grid, P, L, 1, &nu, dt, out);
    int rc = check_args(grid, P, scheme_order, L);
    if (rc != AT_OK) return rc;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(AT_ERR_ARG, "dt must be positive");
    if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(AT_ERR_ARG, "nu must be >= 0");
    const int64_t N = grid->n[0];
    const double dx = grid->length[0] / (double)N;
    const double lim = scheme_order == 2 ? 0.5 : 0.375;   // forward Euler, pure diffusion
    if (!(grid->flags & AT_FLAG_ALLOW_UNSTABLE) && nu * dt / (dx * dx) > lim)
        return fail(AT_ERR_UNSTABLE, "nu*dt/dx^2 = %g exceeds %g", nu * dt / (dx * dx), lim);
    const int w = grid->dtype == AT_F64 ? 8 : 4;
    const int s = scheme_order / 2 + 1;
    const int T = ring_slots(L, s);
    const bool comp = (grid->flags & AT_FLAG_COMPENSATED) != 0;
    if (comp && (w != 4 || (grid->flags & AT_FLAG_VISCOUS_FP64)))
        return fail(AT_ERR_ARG, "AT_FLAG_COMPENSATED needs FP32 state and excludes AT_FLAG_VISCOUS_FP64");
    const Layout lay = layout(N, P, w, L, T, 0, comp);
    if (!grid->workspace) return fail(AT_ERR_ARG, "workspace is NULL");
    if (grid->workspace_bytes < lay.total)
        return fail(AT_ERR_ARG, "workspace too small: %zu < %zu", grid->workspace_bytes, lay.total);
    if (reinterpret_cast<uintptr_t>(grid->workspace) % 256 != 0)
        return fail(AT_ERR_ARG, "workspace must be 256-byte aligned");

    int dev = 0, sms = 0, coop = 0, smem_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop) return fail(AT_ERR_RESIDENCY, "device does not support cooperative launch");

    at_solver *h = new (std::nothrow) at_solver();
    if (!h) return fail(AT_ERR_ARG, "out of host memory");
    h->g = *grid;
    if (h->g.timeout_ns <= 0) h->g.timeout_ns = 1000000000ll;
    h->N = N; h->P = P; h->M = N / P;
    h->order = scheme_order; h->L = L; h->R = scheme_order / 2; h->s = s; h->T = T; h->w = w;
    h->nu = nu; h->dt = dt; h->dx = dx;
    h->lay = lay;
    h->ws = static_cast<unsigned char *>(grid->workspace);
    h->stream = static_cast<cudaStream_t>(grid->stream);
    h->device = dev; h->sm_count = sms; h->smem_optin = smem_optin;
    h->batch = false; h->n_inst = 0; h->lmin = L; h->dim = 1; h->K = 1;
    h->comp = comp;
    h->v64 = !comp && viscous_fp64(w, scheme_order, (uint32_t)grid->flags, nu * dt / (dx * dx));

    pick_kernels(w, scheme_order, h->M, grid->forcing_amp != 0.0, h->v64, h->comp, &h->kernel, &h->init_kernel,
                 &h->kernel_bs);

    // launch shape: by default as many CTAs of kWarps processing elements
    // (warps) as can be resident, at most one PE per subdomain; `stages`
    // tile buffers per PE, fewer if shared memory is short
    const int sb = grid->steps_per_pass > 0 ? grid->steps_per_pass : 1;
    int stages = grid->stages > 0 ? grid->stages : 3;
    if (stages < atk::kMinStages) stages = atk::kMinStages;
    int rc2 = launch_shape(h->M, w, P, tab_size(h->M, w, grid->forcing_amp != 0.0, false, comp), grid->max_ctas,
                           stages, sms, smem_optin, h->kernel, &h->G, &h->stages, &h->sl, &h->smem, &h->smax);
    if (rc2 != AT_OK) { delete h; return rc2; }
    prepare_bs(h);
    h->sb = sb;
    h->step = 0;
    h->has_state = false;
    *out = h;
    return AT_OK;
}

static atk::Params make_params(const at_solver *h)
{
    atk::Params p{};
    p.u = h->ws + h->lay.u;
    p.ring = h->ws + h->lay.ring;
    p.flag = reinterpret_cast<unsigned long long *>(h->ws + h->lay.flag);
    p.ctrl = reinterpret_cast<int *>(h->ws + h->lay.ctrl);
    p.hist = reinterpret_cast<unsigned long long *>(h->ws + h->lay.hist);
    p.gbar = reinterpret_cast<unsigned long long *>(h->ws + h->lay.gbar);
    if (h->comp) p.ur = h->ws + h->lay.ur;
    p.strip = h->ws + h->lay.strip;
    p.ntiles = h->P;
    p.ktile = 1;
    if (h->batch) {
        p.tiles = reinterpret_cast<const int4 *>(h->ws + h->lay.tiles);   // one subdomain per tile
        p.sub_order = reinterpret_cast<const int *>(h->ws + h->lay.order);
        p.ktile = h->K;
        p.bsub = reinterpret_cast<const atk::BatchSub *>(h->ws + h->lay.bsub);
        p.binst = reinterpret_cast<const atk::BatchInst *>(h->ws + h->lay.binst);
    }
    p.N = h->N; p.P = h->P; p.M = h->M;
    p.L = h->L; p.T = h->T;
    p.per_sub = (h->g.flags & AT_FLAG_PER_SUBDOMAIN_DELAY) ? 1 : 0;
    p.seed = h->g.seed;
    if (h->order == 2) {
        p.cA = h->dt / (2.0 * h->dx);
        p.cB = h->nu * h->dt / (h->dx * h->dx);
    } else {
        p.cA = h->dt / (12.0 * h->dx);
        p.cB = h->nu * h->dt / (12.0 * h->dx * h->dx);
    }
    p.dtA = h->dt * h->g.forcing_amp;
    p.x0 = h->g.origin[0];
    p.dx = h->dx;
    p.G = h->G;
    p.E = h->G * atk::kWarps;
    p.stages = h->stages;
    p.smax = h->smax;
    p.bar_off = h->sl.bar_off;
    p.hist_off = h->sl.hist_off;
    p.raw_off = h->sl.raw_off;
    p.stage_off = h->sl.stage_off;
    p.stage_bytes = h->sl.stage_bytes;
    p.tab_off = h->sl.tab_off;
    p.sb = 1;
    p.alt = 0;
    p.timeout_ns = h->g.timeout_ns;
    p.skip_publish = (h->g.flags & AT_FLAG_TEST_SKIP_PUBLISH) ? 1 : 0;
    p.skip_step = h->g.test_skip_step;
    return p;
}

int at_set_state(at_solver *h, const void *u)
{
    g_err[0] = 0;
    if (!h || !u) return fail(AT_ERR_ARG, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(h->ws + h->lay.u, u, (size_t)h->N * h->w, cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(state)");
    if (h->dim == 3) {
        atk::Params3 p = make_params3(h);
        void *args[] = {&p};
        const long long work = h->P * 6 * h->nf * h->d3.face_words;
        const int blocks = (int)((work + 255) / 256 < 4096 ? (work + 255) / 256 : 4096);
        e = cudaLaunchKernel(h->init_kernel, dim3(blocks), dim3(256), args, 0, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "launch at_init3d");
        h->step = 0;
        h->flags_E = 0;
        h->has_state = true;
        return AT_OK;
    }
    e = cudaMemsetAsync(h->ws + h->lay.ring, 0, (size_t)h->T * h->P * 2 * atk::kRingEntry, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(ring)");
    if (h->comp) {
        e = cudaMemsetAsync(h->ws + h->lay.ur, 0, (size_t)h->N * h->w, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(error words)");
    }
    atk::Params p = make_params(h);
    void *args[] = {&p};
    const int blocks = (int)((h->P + 255) / 256 < 1024 ? (h->P + 255) / 256 : 1024);
    e = cudaLaunchKernel(h->init_kernel, dim3(blocks), dim3(256), args, 0, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch at_init");
    h->step = 0;
    h->flags_E = 0;
    h->has_state = true;
    return AT_OK;
}

// Levels per pass of the blocked synchronous mode (AT_SYNC with
// steps_per_pass > 1): the largest count up to the solver's steps_per_pass
// whose edge strips (R x count points, rounded up to a multiple of 4) fit the
// strip entry (16 words and 64 bytes) and lie within one subdomain.  The
// compensated state is stepped one level per pass.
static int sync_pass_len(const at_solver *h)
{
    if (h->comp) return 1;
    int sb = h->sb;
    while (sb > 1) {
        const int64_t words = (int64_t)(h->R * sb + 3) / 4 * 4;
        if (words <= 16 && words * h->w <= atk::kStripBytes && words <= h->M) break;
        --sb;
    }
    return sb < 1 ? 1 : sb;
}

static int strip_words(const at_solver *h, int sb) { return (h->R * sb + 3) / 4 * 4; }

static int step_impl(at_solver *h, int64_t n_steps, int delay_mode, int8_t *delays, void *levels, int64_t depth)
{
    if (!h) return fail(AT_ERR_ARG, "NULL handle");
    if (!h->has_state) return fail(AT_ERR_STATE, "at_step before at_set_state");
    if (n_steps < 0) return fail(AT_ERR_ARG, "n_steps < 0");
    if (delay_mode < AT_SYNC || delay_mode > AT_REPLAY) return fail(AT_ERR_ARG, "bad delay_mode %d", delay_mode);
    if (delay_mode == AT_REPLAY && !delays) return fail(AT_ERR_ARG, "AT_REPLAY needs a delays array");
    if (n_steps == 0) return AT_OK;
    if (h->dim == 3) {
        if (levels) return fail(AT_ERR_ARG, "level output is for 1D solvers");
        atk::Params3 p = make_params3(h);
        p.mode = delay_mode;
        p.delays = delays;
        p.n_steps = n_steps;
        // free-running passes of several levels: the blocked kernel
        const bool blk = delay_mode == AT_FREE && h->kernel_b3 != nullptr;
        p.sb = blk ? h->sb : 1;
        if (blk) { p.G = h->G_b3; p.stages = h->stages_b3; }
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(blk ? h->G_b3 : h->G);
        cfg.blockDim = dim3(blk ? atk::kThreads3b : h->nt3);
        cfg.dynamicSmemBytes = (size_t)(blk ? h->smem_b3 : h->smem);
        cfg.stream = h->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void *args[] = {&p, &h->tmap};
        const cudaError_t e = cudaLaunchKernelExC(&cfg, blk ? h->kernel_b3 : h->kernel, args);
        if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of at_stepper3d");
        h->step += n_steps;
        return AT_OK;
    }
    atk::Params p = make_params(h);
    p.mode = delay_mode;
    p.delays = delays;
    p.n_steps = n_steps;
    p.sb = levels ? 1 : delay_mode == AT_FREE ? h->sb : (delay_mode == AT_SYNC && h->bs_ok) ? sync_pass_len(h) : 1;
    // blocked free-running passes alternate their sweep direction; the
    // blocked synchronous passes (a grid barrier before each) need not
    p.alt = (p.sb > 1 && delay_mode == AT_FREE) ? 1 : 0;
    p.strip_words = strip_words(h, p.sb);
    if (h->batch && h->K > 1 && (delay_mode == AT_FREE || delay_mode == AT_SYNC)) {
        // multi-subdomain tiles (the faces between a tile's subdomains at delay 0)
        p.tiles = reinterpret_cast<const int4 *>(h->ws + h->lay.tiles) + h->P;
        p.ntiles = h->ntiles_k;
    }
    p.levels = levels;
    p.levels_depth = depth;
    const cudaError_t e = launch_stepper(h, &p, (delay_mode == AT_SYNC && p.sb > 1) ? h->kernel_bs : h->kernel);
    if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of at_stepper");
    h->step += n_steps;
    return AT_OK;
}

int at_step(at_solver *h, int64_t n_steps, int delay_mode, int8_t *delays)
{
    g_err[0] = 0;
    return step_impl(h, n_steps, delay_mode, delays, nullptr, 0);
}

int at_step_levels(at_solver *h, int64_t n_steps, int delay_mode, int8_t *delays, void *levels, int64_t depth)
{
    g_err[0] = 0;
    if (!levels || depth < 1) return fail(AT_ERR_ARG, "at_step_levels needs a levels array and depth >= 1");
    return step_impl(h, n_steps, delay_mode, delays, levels, depth);
}

int at_set_history(at_solver *h, const void *levels, int64_t depth, int64_t level)
{
    g_err[0] = 0;
    if (!h || !levels) return fail(AT_ERR_ARG, "NULL argument");
    if (h->dim == 3) return fail(AT_ERR_ARG, "at_set_history is for 1D solvers");
    if (h->comp) return fail(AT_ERR_ARG, "at_set_history does not cover the compensated state");
    if (level < 0) return fail(AT_ERR_ARG, "level < 0");
    const int64_t need = level + 1 < h->L + h->s ? level + 1 : h->L + h->s;
    if (depth < need) return fail(AT_ERR_ARG, "depth %lld holds fewer than the %lld levels needed", (long long)depth,
                                  (long long)need);
    const unsigned char *lv = static_cast<const unsigned char *>(levels);
    cudaError_t e = cudaMemcpyAsync(h->ws + h->lay.u, lv + (size_t)(level % depth) * h->N * h->w, (size_t)h->N * h->w,
                                    cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(level)");
    atk::Params p = make_params(h);
    const long long lo = level - need + 1;
    void *kern = h->w == 8 ? atk_restore_kernel_f64(h->order) : atk_restore_kernel_f32(h->order);
    const void *lv_ptr = levels;
    long long depth_ll = depth, lo_ll = lo, level_ll = level;
    void *args[] = {&p, (void *)&lv_ptr, &depth_ll, &lo_ll, &level_ll};
    const long long work = h->P * need;
    const int blocks = (int)((work + 255) / 256 < 1024 ? (work + 255) / 256 : 1024);
    e = cudaLaunchKernel(kern, dim3(blocks), dim3(256), args, 0, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch at_restore");
    h->step = level;
    h->flags_E = 0;
    h->has_state = true;
    return AT_OK;
}

static int read_status(at_solver *h)
{
    int ctrl[atk::kCtrlWords];
    cudaError_t e = cudaMemcpyAsync(ctrl, h->ws + h->lay.ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(status)");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (ctrl[atk::kCtrlStatus] == atk::kStatusTimeout)
        return fail(AT_ERR_TIMEOUT, "device wait timed out (cta %d, where %d, step %d, neighbour %d)",
                    ctrl[atk::kCtrlCta], ctrl[atk::kCtrlWhere], ctrl[atk::kCtrlStep], ctrl[atk::kCtrlNb]);
    if (ctrl[atk::kCtrlStatus] != 0) return fail(AT_ERR_CUDA, "device status %d", ctrl[atk::kCtrlStatus]);
    return AT_OK;
}

int at_state(at_solver *h, void *dst)
{
    g_err[0] = 0;
    if (!h || !dst) return fail(AT_ERR_ARG, "NULL argument");
    if (!h->has_state) return fail(AT_ERR_STATE, "at_state before at_set_state");
    cudaError_t e = cudaMemcpyAsync(dst, h->ws + h->lay.u, (size_t)h->N * h->w, cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(state out)");
    return read_status(h);
}

int at_state_error(at_solver *h, void *dst)
{
    g_err[0] = 0;
    if (!h || !dst) return fail(AT_ERR_ARG, "NULL argument");
    if (!h->comp) return fail(AT_ERR_ARG, "at_state_error needs a compensated state (AT_FLAG_COMPENSATED)");
    if (!h->has_state) return fail(AT_ERR_STATE, "at_state_error before at_set_state");
    cudaError_t e = cudaMemcpyAsync(dst, h->ws + h->lay.ur, (size_t)h->N * h->w, cudaMemcpyDefault, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(error words out)");
    return read_status(h);
}

int at_status(at_solver *h)
{
    g_err[0] = 0;
    if (!h) return fail(AT_ERR_ARG, "NULL handle");
    return read_status(h);
}

int at_delay_stats(at_solver *h, int64_t *hist, double *mean_k, double *mean_k2)
{
    g_err[0] = 0;
    if (!h) return fail(AT_ERR_ARG, "NULL handle");
    unsigned long long cnt[atk::kMaxL + 1] = {0};
    cudaError_t e = cudaMemcpyAsync(cnt, h->ws + h->lay.hist, (size_t)(h->L + 1) * 8, cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(hist)");
    const int rc = read_status(h);
    double tot = 0, m1 = 0, m2 = 0;
    for (int k = 0; k <= h->L; ++k) {
        if (hist) hist[k] = (int64_t)cnt[k];
        tot += (double)cnt[k];
        m1 += (double)k * (double)cnt[k];
        m2 += (double)k * k * (double)cnt[k];
    }
    if (mean_k) *mean_k = tot > 0 ? m1 / tot : 0.0;
    if (mean_k2) *mean_k2 = tot > 0 ? m2 / tot : 0.0;
    return rc;
}

int at_get_info(const at_solver *h, at_info *info)
{
    if (!h || !info) return fail(AT_ERR_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    // (3D: M is the points per subdomain, sub[0] sub[1] sub[2])
    info->N = h->N; info->P = h->P; info->M = h->M;
    info->order = h->order; info->L = h->L; info->R = h->R; info->s = h->s; info->T = h->T;
    info->ctas = h->G; info->threads = h->dim == 3 ? h->nt3 : atk::kThreads; info->stages = h->stages;
    info->smem_bytes = h->smem; info->step = h->step; info->sm_count = h->sm_count;
    info->dtype = h->g.dtype; info->steps_per_pass = h->sb;
    info->viscous_fp64 = h->v64 ? 1 : 0;
    info->tile_subdomains = h->batch ? h->K : 1;
    if (h->dim == 3 && h->kernel_b3) {
        // 3D with several levels per pass: the blocked AT_FREE kernel's shape
        info->ctas = h->G_b3; info->threads = atk::kThreads3b; info->stages = h->stages_b3;
        info->smem_bytes = h->smem_b3;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (h->has_state && cudaStreamIsCapturing(h->stream, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
        long long n0 = 0;
        cudaError_t e = cudaMemcpyAsync(&n0, h->ws + h->lay.ctrl + 4 * atk::kCtrlN0, sizeof(n0),
                                        cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "reading the level of the state");
        info->step = n0;
    }
    return AT_OK;
}

int at_destroy(at_solver *h)
{
    delete h;
    return AT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Ensembles
// ---------------------------------------------------------------------------
namespace {

struct BatchDims {
    int64_t N, P;
    int Lmax, Lmin;
};

int check_batch(const at_grid *g, int64_t n_inst, const at_instance *inst, int64_t M, int order, BatchDims *d)
{
    if (!g) return fail(AT_ERR_ARG, "grid is NULL");
    if (g->dim != 1) return fail(AT_ERR_ARG, "dim must be 1");
    if (g->dtype != AT_F64 && g->dtype != AT_F32) return fail(AT_ERR_ARG, "dtype must be AT_F64 or AT_F32");
    if (g->forcing_amp != 0.0) return fail(AT_ERR_ARG, "ensembles are unforced (forcing_amp must be 0)");
    if (order != 2 && order != 4) return fail(AT_ERR_ARG, "scheme_order must be 2 or 4");
    if (M % 4 != 0 || M < 4 || M > atk::kMaxM)
        return fail(AT_ERR_ARG, "M must be a multiple of 4 in 4..%d (M=%lld)", atk::kMaxM, (long long)M);
    if (n_inst <= 0 || !inst) return fail(AT_ERR_ARG, "no instances");
    d->N = 0;
    d->Lmax = 0;
    d->Lmin = atk::kMaxL;
    const double lim = order == 2 ? 0.5 : 0.375;
    for (int64_t j = 0; j < n_inst; ++j) {
        const at_instance &a = inst[j];
        if (a.n <= 0 || a.n % M != 0)
            return fail(AT_ERR_ARG, "instance %lld: n=%lld is not a positive multiple of M=%lld", (long long)j,
                        (long long)a.n, (long long)M);
        if (a.L < 0 || a.L > atk::kMaxL) return fail(AT_ERR_ARG, "instance %lld: L must be in 0..%d", (long long)j,
                                                     atk::kMaxL);
        if (a.bc != AT_BC_PERIODIC && a.bc != AT_BC_EXACT_TANH)
            return fail(AT_ERR_ARG, "instance %lld: bad bc %d", (long long)j, a.bc);
        if (!(a.length > 0.0) || !std::isfinite(a.length) || !std::isfinite(a.origin))
            return fail(AT_ERR_ARG, "instance %lld: length must be positive", (long long)j);
        if (!(a.dt > 0.0) || !std::isfinite(a.dt)) return fail(AT_ERR_ARG, "instance %lld: dt must be positive",
                                                                (long long)j);
        if (!(a.nu >= 0.0) || !std::isfinite(a.nu)) return fail(AT_ERR_ARG, "instance %lld: nu must be >= 0",
                                                                 (long long)j);
        if (a.bc == AT_BC_EXACT_TANH && !(a.nu > 0.0))
            return fail(AT_ERR_ARG, "instance %lld: exact tanh boundary values need nu > 0", (long long)j);
        const double dx = a.length / (double)a.n;
        if (!(g->flags & AT_FLAG_ALLOW_UNSTABLE) && a.nu * a.dt / (dx * dx) > lim)
            return fail(AT_ERR_UNSTABLE, "instance %lld: nu*dt/dx^2 = %g exceeds %g", (long long)j,
                        a.nu * a.dt / (dx * dx), lim);
        d->N += a.n;
        if (a.L > d->Lmax) d->Lmax = a.L;
        if (a.L < d->Lmin) d->Lmin = a.L;
    }
    d->P = d->N / M;
    if (d->P >= (1LL << 31)) return fail(AT_ERR_ARG, "at most 2^31 - 1 subdomains");
    if (g->steps_per_pass < 0 || g->steps_per_pass > d->Lmax + 1)
        return fail(AT_ERR_ARG, "steps_per_pass must be in 0..max L + 1, got %d", g->steps_per_pass);
    const int K = g->tile_subdomains > 1 ? g->tile_subdomains : 1;
    if (g->tile_subdomains < 0 || (K != 1 && K != 2 && K != 4))
        return fail(AT_ERR_ARG, "tile_subdomains must be 0, 1, 2 or 4, got %d", g->tile_subdomains);
    if (K > 1 && (M != 128 && M != 256 && M != 512))
        return fail(AT_ERR_ARG, "tile_subdomains > 1 needs M = 128, 256 or 512 (M=%lld)", (long long)M);
    if ((int64_t)K * M > atk::kMaxM)
        return fail(AT_ERR_ARG, "tile_subdomains x M must be <= %d", atk::kMaxM);
    return AT_OK;
}

}  // namespace

extern "C" {

size_t at_batch_workspace_bytes(const at_grid *grid, int64_t n_inst, const at_instance *inst, int64_t M,
                                int scheme_order)
{
    BatchDims d{};
    if (check_batch(grid, n_inst, inst, M, scheme_order, &d) != AT_OK) return 0;
    const int w = grid->dtype == AT_F64 ? 8 : 4;
    const int s = scheme_order / 2 + 1;
    return layout(d.N, d.P, w, d.Lmax, ring_slots(d.Lmax, s), n_inst, (grid->flags & AT_FLAG_COMPENSATED) != 0).total;
}

int at_create_batch(const at_grid *grid, int64_t n_inst, const at_instance *inst, int64_t M, int scheme_order,
                    at_solver **out)
{
    g_err[0] = 0;
    if (!out) return fail(AT_ERR_ARG, "out is NULL");
    *out = nullptr;
    BatchDims d{};
    int rc = check_batch(grid, n_inst, inst, M, scheme_order, &d);
    if (rc != AT_OK) return rc;
    const int w = grid->dtype == AT_F64 ? 8 : 4;
    const int s = scheme_order / 2 + 1;
    const int T = ring_slots(d.Lmax, s);
    const bool comp = (grid->flags & AT_FLAG_COMPENSATED) != 0;
    if (comp && w != 4) return fail(AT_ERR_ARG, "AT_FLAG_COMPENSATED needs FP32 state");
    const Layout lay = layout(d.N, d.P, w, d.Lmax, T, n_inst, comp);
    if (!grid->workspace) return fail(AT_ERR_ARG, "workspace is NULL");
    if (grid->workspace_bytes < lay.total)
        return fail(AT_ERR_ARG, "workspace too small: %zu < %zu", grid->workspace_bytes, lay.total);
    if (reinterpret_cast<uintptr_t>(grid->workspace) % 256 != 0)
        return fail(AT_ERR_ARG, "workspace must be 256-byte aligned");

    int dev = 0, sms = 0, coop = 0, smem_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop) return fail(AT_ERR_RESIDENCY, "device does not support cooperative launch");

    // subdomain and instance records
    std::vector<atk::BatchSub> sub((size_t)d.P);
    std::vector<atk::BatchInst> ins((size_t)n_inst);
    int64_t p0 = 0;
    for (int64_t j = 0; j < n_inst; ++j) {
        const at_instance &a = inst[j];
        const double dx = a.length / (double)a.n;
        const int64_t Pi = a.n / M;
        atk::BatchInst &bi = ins[(size_t)j];
        bi = atk::BatchInst{};
        bi.x0 = a.origin; bi.dx = dx; bi.dt = a.dt; bi.nu = a.nu;
        bi.ta = a.tanh_a; bi.tc = a.tanh_c; bi.txc = a.tanh_xc;
        const bool periodic = a.bc == AT_BC_PERIODIC;
        for (int64_t lp = 0; lp < Pi; ++lp) {
            atk::BatchSub &b = sub[(size_t)(p0 + lp)];
            b = atk::BatchSub{};
            if (scheme_order == 2) {
                b.cA = a.dt / (2.0 * dx);
                b.cB = a.nu * a.dt / (dx * dx);
            } else {
                b.cA = a.dt / (12.0 * dx);
                b.cB = a.nu * a.dt / (12.0 * dx * dx);
            }
            b.seed = a.seed;
            b.L = a.L;
            b.lp = (int)lp;
            b.Pi = (int)Pi;
            b.inst = (int)j;
            b.left = lp > 0 ? p0 + lp - 1 : (periodic ? p0 + Pi - 1 : -1);
            b.right = lp < Pi - 1 ? p0 + lp + 1 : (periodic ? p0 : -1);
        }
        p0 += Pi;
    }
    unsigned char *ws = static_cast<unsigned char *>(grid->workspace);
    cudaStream_t st = static_cast<cudaStream_t>(grid->stream);
    e = cudaMemcpyAsync(ws + lay.bsub, sub.data(), sub.size() * sizeof(atk::BatchSub), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + lay.binst, ins.data(), ins.size() * sizeof(atk::BatchInst), cudaMemcpyHostToDevice,
                            st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "copying the ensemble tables");

    at_solver *h = new (std::nothrow) at_solver();
    if (!h) return fail(AT_ERR_ARG, "out of host memory");
    h->g = *grid;
    if (h->g.timeout_ns <= 0) h->g.timeout_ns = 1000000000ll;
    h->N = d.N; h->P = d.P; h->M = M;
    h->order = scheme_order; h->L = d.Lmax; h->R = scheme_order / 2; h->s = s; h->T = T; h->w = w;
    h->nu = 0; h->dt = 0; h->dx = 0;
    h->lay = lay;
    h->ws = ws;
    h->stream = st;
    h->device = dev; h->sm_count = sms; h->smem_optin = smem_optin;
    h->batch = true; h->n_inst = n_inst; h->lmin = d.Lmin;
    h->comp = comp;
    h->bsub_host = std::move(sub);
    h->inst_host.assign(inst, inst + n_inst);
    rc = set_tile_plan(h, grid->tile_subdomains > 1 ? grid->tile_subdomains : 1);
    if (rc != AT_OK) { delete h; return rc; }
    h->init_kernel = w == 8 ? atk_init_kernel_f64(scheme_order) : atk_init_kernel_f32(scheme_order);
    int stages = grid->stages > 0 ? grid->stages : 3;
    if (stages < atk::kMinStages) stages = atk::kMinStages;
    rc = launch_shape((int64_t)h->K * M, w, d.P, tab_size(M, w, false, true, comp, h->ntiles_k, h->K), grid->max_ctas,
                      stages, sms, smem_optin, h->kernel, &h->G, &h->stages, &h->sl, &h->smem, &h->smax);
    if (rc != AT_OK) { delete h; return rc; }
    prepare_bs(h);
    h->sb = grid->steps_per_pass > 0 ? grid->steps_per_pass : 1;
    h->step = 0;
    h->has_state = false;
    *out = h;
    return AT_OK;
}

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------
int at_tune(at_solver *h, int64_t n_steps, int delay_mode, at_tune_result *res)
{
    g_err[0] = 0;
    if (!h || !res) return fail(AT_ERR_ARG, "NULL argument");
    if (h->dim == 3) return fail(AT_ERR_ARG, "at_tune is for 1D solvers");
    if (!h->has_state) return fail(AT_ERR_STATE, "at_tune before at_set_state");
    if (n_steps <= 0) return fail(AT_ERR_ARG, "n_steps must be positive");
    if (delay_mode != AT_SYNC && delay_mode != AT_SEEDED && delay_mode != AT_FREE)
        return fail(AT_ERR_ARG, "at_tune times AT_SYNC, AT_SEEDED or AT_FREE");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return fail(AT_ERR_STATE, "at_tune under stream capture");
    std::memset(res, 0, sizeof(*res));
    const int gmax = (int)((h->P + atk::kWarps - 1) / atk::kWarps);

    cudaEvent_t ev[3];
    for (int i = 0; i < 3; ++i) {
        const cudaError_t e = cudaEventCreate(&ev[i]);
        if (e != cudaSuccess) {
            for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    struct Shape {
        int G, stages, sb, K;
    };
    auto apply = [&](const Shape &sh) -> int {
        if (h->batch && sh.K != h->K) {
            const int r = set_tile_plan(h, sh.K);
            if (r != AT_OK) return r;
        }
        // (a tile is one subdomain, except in an ensemble of K-subdomain tiles)
        const int kt = h->batch ? h->K : 1;
        const TabSize tsz = tab_size(h->M, h->w, h->g.forcing_amp != 0.0, h->batch, h->comp, h->ntiles_k, kt);
        int G = 0, st = 0, smem = 0;
        long long smax = 0;
        atk::SmemLayout sl{};
        const int r = launch_shape((int64_t)kt * h->M, h->w, h->P, tsz, sh.G, sh.stages, h->sm_count,
                                   h->smem_optin, h->kernel, &G, &st, &sl, &smem, &smax);
        if (r != AT_OK) return r;
        if (st != sh.stages) return AT_ERR_RESIDENCY;   // did not fit as asked
        h->G = G; h->stages = st; h->sl = sl; h->smem = smem; h->smax = smax; h->sb = sh.sb;
        prepare_bs(h);
        return AT_OK;
    };
    // time of one at_step(n_steps): one untimed launch, best of two timed
    auto time_shape = [&](double *ms) -> int {
        int r = at_step(h, n_steps, delay_mode, nullptr);
        if (r != AT_OK) return r;
        double best = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(ev[0], h->stream);
            r = at_step(h, n_steps, delay_mode, nullptr);
            if (r != AT_OK) return r;
            cudaEventRecord(ev[1], h->stream);
            const cudaError_t e = cudaEventSynchronize(ev[1]);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[0], ev[1]);
            if (t < best) best = t;
        }
        r = read_status(h);
        if (r != AT_OK) return r;
        *ms = best;
        return AT_OK;
    };

    const Shape orig{h->G, h->stages, h->sb, h->batch ? h->K : 1};
    Shape best = orig;
    double best_ms = 0.0;
    int rc = time_shape(&best_ms);
    int tried = 1;
    res->first_ms = best_ms;
    // levels per pass: up to the largest delay bound + 1 (an ensemble's PEs
    // clamp it to their own smallest bound + 1); the synchronous mode keeps
    // one level per pass unless the solver was made for blocked passes
    const int sb_hi = (delay_mode == AT_FREE || (delay_mode == AT_SYNC && h->sb > 1)) ? h->L + 1 : 1;
    // ensembles in AT_FREE / AT_SYNC: subdomains per tile 1, 2, 4 (as the
    // subdomain size allows)
    int k_hi = 1;
    if (h->batch && (delay_mode == AT_FREE || delay_mode == AT_SYNC) &&
        (h->M == 128 || h->M == 256 || h->M == 512))
        k_hi = (int)(atk::kMaxM / h->M) < 4 ? (int)(atk::kMaxM / h->M) : 4;
    for (int K = 1; rc == AT_OK && K <= k_hi; K *= 2) {
        for (int st = atk::kMinStages; rc == AT_OK && st <= 4; ++st) {
            int lastG = -1;
            for (int per_sm = 1; rc == AT_OK && per_sm <= 4; ++per_sm) {
                const int G = per_sm * h->sm_count < gmax ? per_sm * h->sm_count : gmax;
                if (G == lastG) break;
                lastG = G;
                for (int sb = 1; rc == AT_OK && sb <= sb_hi; ++sb) {
                    const Shape sh{G, st, sb, h->batch ? K : 1};
                    if (sh.G == orig.G && sh.stages == orig.stages && sh.sb == orig.sb && sh.K == orig.K) continue;
                    const int ra = apply(sh);
                    if (ra == AT_ERR_CUDA) { rc = ra; break; }
                    if (ra != AT_OK) { g_err[0] = 0; continue; }   // not resident: skip
                    double ms = 0.0;
                    rc = time_shape(&ms);
                    ++tried;
                    if (rc == AT_OK && ms < best_ms) { best_ms = ms; best = sh; }
                }
            }
        }
    }
    for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
    const int rc_apply = apply(rc == AT_OK ? best : orig);
    if (rc != AT_OK) return rc;
    if (rc_apply != AT_OK) return rc_apply;
    res->ctas = h->G;
    res->stages = h->stages;
    res->steps_per_pass = h->sb;
    res->tile_subdomains = h->batch ? h->K : 1;
    res->n_tried = tried;
    res->best_ms = best_ms;
    return AT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpointed forward run and the discrete adjoint
// ---------------------------------------------------------------------------
namespace {

// levels kept per checkpoint: the level itself and the L + s - 1 before it
// (the oldest level the next step's halos read)
int64_t ckpt_levels(const at_solver *h) { return h->L + h->s; }

int64_t n_segments(int64_t n_steps, int64_t interval) { return n_steps <= 0 ? 1 : (n_steps + interval - 1) / interval; }

// adjoint launch: x walks the subdomains, y the 1024-point chunks of one
int adj_grid_x(const at_solver *h) { return (int)(h->P < 16LL * h->sm_count ? h->P : 16LL * h->sm_count); }
int adj_grid_y(const at_solver *h) { return (int)((h->M + atk::kAdjChunk - 1) / atk::kAdjChunk); }
int adj_blocks(const at_solver *h) { return adj_grid_x(h) * adj_grid_y(h); }

struct AdjLayout {
    size_t levels, lam, pend, dnu, bar, kbuf, total;
};

AdjLayout adj_layout(const at_solver *h, int64_t interval)
{
    AdjLayout l{};
    size_t off = 0;
    l.levels = off; off = align_up(off + (size_t)(interval + ckpt_levels(h)) * h->N * h->w, 256);
    l.lam = off;    off = align_up(off + (size_t)h->N * h->w, 256);
    l.pend = off;   off = align_up(off + (size_t)h->T * h->P * 2 * h->R * h->w, 256);
    l.dnu = off;    off = align_up(off + (size_t)adj_blocks(h) * 8, 256);
    l.bar = off;    off = align_up(off + 8, 256);
    l.kbuf = off;   off = align_up(off + (size_t)interval * h->P * 2, 256);
    l.total = off;
    return l;
}

int check_adjoint_args(const at_solver *h, int64_t n_steps, int64_t interval)
{
    if (!h) return fail(AT_ERR_ARG, "NULL handle");
    if (h->batch || h->dim == 3) return fail(AT_ERR_ARG, "the adjoint covers single-domain 1D solvers");
    if (h->comp) return fail(AT_ERR_ARG, "the adjoint does not cover the compensated state");
    if (h->N >= (1LL << 31)) return fail(AT_ERR_ARG, "the adjoint needs N < 2^31");
    if (n_steps < 0) return fail(AT_ERR_ARG, "n_steps < 0");
    if (interval < 1) return fail(AT_ERR_ARG, "interval must be >= 1");
    return AT_OK;
}

}  // namespace

extern "C" {

size_t at_checkpoint_bytes(const at_solver *h, int64_t n_steps, int64_t interval)
{
    if (check_adjoint_args(h, n_steps, interval) != AT_OK) return 0;
    return (size_t)n_segments(n_steps, interval) * (size_t)ckpt_levels(h) * (size_t)h->N * h->w;
}

int at_step_checkpointed(at_solver *h, int64_t n_steps, int delay_mode, int8_t *delays, int64_t interval, void *ckpt)
{
    g_err[0] = 0;
    int rc = check_adjoint_args(h, n_steps, interval);
    if (rc != AT_OK) return rc;
    if (!ckpt) return fail(AT_ERR_ARG, "ckpt is NULL");
    if (!h->has_state || h->step != 0) return fail(AT_ERR_STATE, "at_step_checkpointed starts at level 0 (after at_set_state)");
    const int64_t Dc = ckpt_levels(h), nseg = n_segments(n_steps, interval);
    const size_t lvl = (size_t)h->N * h->w, seg_bytes = (size_t)Dc * lvl;
    unsigned char *ck = static_cast<unsigned char *>(ckpt);
    cudaError_t e = cudaMemsetAsync(ck, 0, seg_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ck, h->ws + h->lay.u, lvl, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint 0");
    for (int64_t seg = 0; seg < nseg; ++seg) {
        const int64_t c = seg * interval;
        const int64_t len = n_steps - c < interval ? n_steps - c : interval;
        int8_t *d = delays ? delays + (size_t)c * h->P * 2 : nullptr;
        if (seg + 1 < nseg) {
            // the next checkpoint starts as a copy of this one, so that it also
            // holds the levels before c when the interval is shorter than Dc
            e = cudaMemcpyAsync(ck + (size_t)(seg + 1) * seg_bytes, ck + (size_t)seg * seg_bytes, seg_bytes,
                                cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "checkpoint copy");
            rc = step_impl(h, len, delay_mode, d, ck + (size_t)(seg + 1) * seg_bytes, Dc);
        } else {
            rc = step_impl(h, len, delay_mode, d, nullptr, 0);
        }
        if (rc != AT_OK) return rc;
    }
    return AT_OK;
}

size_t at_adjoint_workspace_bytes(const at_solver *h, int64_t interval)
{
    if (check_adjoint_args(h, 0, interval) != AT_OK) return 0;
    return adj_layout(h, interval).total;
}

int at_adjoint(at_solver *h, int64_t n_steps, int delay_mode, const int8_t *delays, int64_t interval,
               const void *ckpt, void *adj_ws, size_t adj_ws_bytes, void *lam, double *dnu)
{
    g_err[0] = 0;
    int rc = check_adjoint_args(h, n_steps, interval);
    if (rc != AT_OK) return rc;
    if (!ckpt || !adj_ws || !lam) return fail(AT_ERR_ARG, "NULL argument");
    if (delay_mode != AT_SYNC && delay_mode != AT_SEEDED && delay_mode != AT_REPLAY)
        return fail(AT_ERR_ARG, "the adjoint replays AT_SYNC, AT_SEEDED or AT_REPLAY delays (record AT_FREE ones)");
    if (delay_mode == AT_REPLAY && !delays) return fail(AT_ERR_ARG, "AT_REPLAY needs a delays array");
    const AdjLayout al = adj_layout(h, interval);
    if (adj_ws_bytes < al.total) return fail(AT_ERR_ARG, "adjoint workspace too small: %zu < %zu", adj_ws_bytes, al.total);
    if (reinterpret_cast<uintptr_t>(adj_ws) % 256 != 0) return fail(AT_ERR_ARG, "adjoint workspace must be 256-byte aligned");
    if (!h->has_state) return fail(AT_ERR_STATE, "at_adjoint needs the solver's state to have been set");
    const int64_t Dc = ckpt_levels(h), Dl = interval + Dc, nseg = n_segments(n_steps, interval);
    const size_t lvl = (size_t)h->N * h->w, seg_bytes = (size_t)Dc * lvl;
    unsigned char *ws = static_cast<unsigned char *>(adj_ws);
    const unsigned char *ck = static_cast<const unsigned char *>(ckpt);
    const int G = adj_blocks(h);
    cudaError_t e = cudaMemsetAsync(ws + al.pend, 0, al.dnu - al.pend + (size_t)G * 8, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(adjoint)");

    atk::AdjParams a{};
    a.levels = ws + al.levels;
    a.Dl = Dl;
    a.pend = ws + al.pend;
    a.dnu_part = reinterpret_cast<double *>(ws + al.dnu);
    a.bar = reinterpret_cast<unsigned long long *>(ws + al.bar);
    a.ctrl = reinterpret_cast<int *>(h->ws + h->lay.ctrl);
    a.timeout_ns = h->g.timeout_ns;
    a.N = h->N; a.P = h->P; a.M = h->M;
    a.L = h->L; a.Tp = h->T;
    if (h->order == 2) {
        a.cA = h->dt / (2.0 * h->dx);
        a.cB = h->nu * h->dt / (h->dx * h->dx);
        a.dtdx2 = h->dt / (h->dx * h->dx);
    } else {
        a.cA = h->dt / (12.0 * h->dx);
        a.cB = h->nu * h->dt / (12.0 * h->dx * h->dx);
        a.dtdx2 = h->dt / (12.0 * h->dx * h->dx);
    }
    a.cAf = (float)a.cA; a.cBf = (float)a.cB; a.dtdx2f = (float)a.dtdx2;
    // one cooperative launch per interval: every block resident.  With one
    // block per subdomain (M <= 1024 points, every subdomain's block
    // resident) the variant that keeps lambda in registers and loads the next
    // level's lambda-free data before the grid barrier; else blocks walk the
    // subdomains
    void *kern = atk_adjoint_own_kernel(h->w, h->order);
    int threads = atk::kAdjOwnThreads;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(adjoint)");
    int gy = 1, gx = (int)h->P;
    // (FP32, order 2: the variant's per-thread data fits its registers there)
    const bool own = h->w == 4 && h->order == 2 && h->M <= atk::kAdjOwnChunk &&
                     h->P <= (int64_t)occ * h->sm_count && h->P <= adj_blocks(h);
    if (!own) {
        kern = atk_adjoint_kernel(h->w, h->order);
        threads = atk::kAdjThreads;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(adjoint)");
        gy = adj_grid_y(h);
        gx = adj_grid_x(h);
        if ((int64_t)gx * gy > (int64_t)occ * h->sm_count) gx = (int)((int64_t)occ * h->sm_count / gy);
        if (gx < 1) return fail(AT_ERR_RESIDENCY, "adjoint: %d blocks per subdomain cannot be co-resident", gy);
    }
    unsigned char *cur = static_cast<unsigned char *>(lam), *other = ws + al.lam;
    for (int64_t seg = nseg - 1; seg >= 0; --seg) {
        const int64_t c = seg * interval;
        const int64_t end = n_steps - c < interval ? n_steps : c + interval;
        // levels c-Dc+1 .. c from the checkpoint, then c+1 .. end recomputed
        for (int64_t l = (c - Dc + 1 > 0 ? c - Dc + 1 : 0); l <= c; ++l) {
            e = cudaMemcpyAsync(ws + al.levels + (size_t)(l % Dl) * lvl, ck + (size_t)seg * seg_bytes + (size_t)(l % Dc) * lvl,
                                lvl, cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "restoring levels");
        }
        rc = at_set_history(h, ck + (size_t)seg * seg_bytes, Dc, c);
        if (rc != AT_OK) return rc;
        // the recomputation replays the given delays or records the ones it
        // draws; the adjoint reads them from there
        int8_t *d = delay_mode == AT_REPLAY ? const_cast<int8_t *>(delays) + (size_t)c * h->P * 2
                                            : reinterpret_cast<int8_t *>(ws + al.kbuf);
        rc = step_impl(h, end - c, delay_mode, d, ws + al.levels, Dl);
        if (rc != AT_OK) return rc;
        if (end == c) continue;
        a.delays = d;
        a.k_level = c;
        a.n_hi = end;
        a.n_lo = c;
        a.lam_a = cur;
        a.lam_b = other;
        e = cudaMemsetAsync(a.bar, 0, 8, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(adjoint barrier)");
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(gx, gy);
        cfg.blockDim = dim3(threads);
        cfg.stream = h->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void *args[] = {&a};
        e = cudaLaunchKernelExC(&cfg, kern, args);
        if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of at_adjoint_interval");
        if ((end - c) & 1) { unsigned char *t = cur; cur = other; other = t; }
    }
    if (cur != lam) {
        e = cudaMemcpyAsync(lam, cur, lvl, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(lambda)");
    }
    std::vector<double> part((size_t)G);
    e = cudaMemcpyAsync(part.data(), ws + al.dnu, (size_t)G * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(dnu)");
    rc = read_status(h);
    if (rc != AT_OK) return rc;
    double sum = 0.0;
    for (int b = 0; b < G; ++b) sum += part[(size_t)b];
    if (dnu) *dnu = sum;
    return AT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point (at_step_noalloc).
//
// Some callers cannot allocate device memory: a plug-in living inside a host
// application that owns every byte of device memory and gives it only the
// state buffer, code with a hard device-memory budget, or a loop that must
// never reach the CUDA allocator.  at_step_noalloc serves them by running the
// same persistent kernel with its scratch -- ring buffers, progress flags,
// control block, delay counters and barrier counter -- in the fixed array
// below, which every GPU that loads this library keeps until the process
// exits.  The caller still passes the state (input and output) and, if used,
// the delay array.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[AT_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the current device's context.  In
// host code the array's name is only a host-side stand-in, so the address is
// looked up with the device current -- on every call, not cached: after a
// context is torn down and created again (cudaDeviceReset, a primary-context
// reset) the module is loaded anew and the array may sit elsewhere, and a
// cached address would then point into memory that is no longer the array.
int noalloc_scratch_address(unsigned char **out)
{
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch array)");
    *out = static_cast<unsigned char *>(ptr);
    return AT_OK;
}

}  // namespace

extern "C" int at_step_noalloc(const at_grid *grid, int64_t P, int scheme_order, int L, double nu, double dt,
                               void *u, int64_t n_steps, int delay_mode, int8_t *delays)
{
    g_err[0] = 0;
    if (grid && grid->dim != 1) return fail(AT_ERR_ARG, "at_step_noalloc is for 1D grids");
    int rc = check_args(grid, P, scheme_order, L);
    if (rc != AT_OK) return rc;
    if (!u) return fail(AT_ERR_ARG, "u is NULL");
    if (reinterpret_cast<uintptr_t>(u) % 16 != 0) return fail(AT_ERR_ARG, "u must be 16-byte aligned");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(AT_ERR_ARG, "dt must be positive");
    if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(AT_ERR_ARG, "nu must be >= 0");
    if (n_steps < 0) return fail(AT_ERR_ARG, "n_steps < 0");
    if (delay_mode < AT_SYNC || delay_mode > AT_REPLAY) return fail(AT_ERR_ARG, "bad delay_mode %d", delay_mode);
    if (delay_mode == AT_REPLAY && !delays) return fail(AT_ERR_ARG, "AT_REPLAY needs a delays array");
    if (grid->steps_per_pass > 1)
        return fail(AT_ERR_ARG, "at_step_noalloc runs one level per pass (steps_per_pass must be 0 or 1, got %d)",
                    grid->steps_per_pass);
    if (grid->flags & AT_FLAG_COMPENSATED) return fail(AT_ERR_ARG, "at_step_noalloc has no compensated state");
    const int64_t N = grid->n[0];
    const double dx = grid->length[0] / (double)N;
    const double lim = scheme_order == 2 ? 0.5 : 0.375;
    if (!(grid->flags & AT_FLAG_ALLOW_UNSTABLE) && nu * dt / (dx * dx) > lim)
        return fail(AT_ERR_UNSTABLE, "nu*dt/dx^2 = %g exceeds %g", nu * dt / (dx * dx), lim);
    const int w = grid->dtype == AT_F64 ? 8 : 4;
    const int s = scheme_order / 2 + 1;
    const int T = ring_slots(L, s);
    const Layout lay = layout(0, P, w, L, T, 0, false, false);   // scratch only: the state is the caller's
    if (lay.total > (size_t)AT_NOALLOC_SCRATCH_BYTES)
        return fail(AT_ERR_ARG,
                    "at_step_noalloc: P=%lld, L=%d, order %d need %zu bytes of scratch, more than the "
                    "fixed %zu-byte array (use at_create with a workspace)",
                    (long long)P, L, scheme_order, lay.total, (size_t)AT_NOALLOC_SCRATCH_BYTES);

    int dev = 0, sms = 0, coop = 0, smem_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop) return fail(AT_ERR_RESIDENCY, "device does not support cooperative launch");
    unsigned char *scratch = nullptr;
    rc = noalloc_scratch_address(&scratch);
    if (rc != AT_OK) return rc;

    at_solver h{};   // on the stack: nothing is allocated, on the host or on the device
    h.g = *grid;
    if (h.g.timeout_ns <= 0) h.g.timeout_ns = 1000000000ll;
    h.N = N; h.P = P; h.M = N / P;
    h.order = scheme_order; h.L = L; h.R = scheme_order / 2; h.s = s; h.T = T; h.w = w;
    h.nu = nu; h.dt = dt; h.dx = dx;
    h.lay = lay;
    h.ws = scratch;
    h.stream = static_cast<cudaStream_t>(grid->stream);
    h.device = dev; h.sm_count = sms; h.smem_optin = smem_optin;
    h.batch = false; h.n_inst = 0; h.lmin = L; h.K = 1;
    h.comp = false;
    h.v64 = viscous_fp64(w, scheme_order, (uint32_t)grid->flags, nu * dt / (dx * dx));
    pick_kernels(w, scheme_order, h.M, grid->forcing_amp != 0.0, h.v64, false, &h.kernel, &h.init_kernel);
    int stages = grid->stages > 0 ? grid->stages : 3;
    if (stages < atk::kMinStages) stages = atk::kMinStages;
    rc = launch_shape(h.M, w, P, tab_size(h.M, w, grid->forcing_amp != 0.0, false), grid->max_ctas, stages, sms,
                      smem_optin, h.kernel, &h.G, &h.stages, &h.sl, &h.smem, &h.smax);
    if (rc != AT_OK) return rc;
    h.sb = 1;

    // Every call starts from zeroed ring buffers, flags, status and counters:
    // the array still holds whatever the previous call left in it.
    atk::Params p = make_params(&h);
    p.u = u;
    e = cudaMemsetAsync(scratch + lay.ring, 0, lay.total - lay.ring, h.stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(scratch)");
    void *args[] = {&p};
    const int blocks = (int)((P + 255) / 256 < 1024 ? (P + 255) / 256 : 1024);
    e = cudaLaunchKernel(h.init_kernel, dim3(blocks), dim3(256), args, 0, h.stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch at_init");
    if (n_steps > 0) {
        p.mode = delay_mode;
        p.delays = delays;
        p.n_steps = n_steps;
        p.sb = 1;
        e = launch_stepper(&h, &p, h.kernel);
        if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of at_stepper");
    }
    return read_status(&h);
}

// ---------------------------------------------------------------------------
// The 3D system of Eq. BS and its moments
// ---------------------------------------------------------------------------
namespace {

// per-block sums of q and q^2 of every field (FP64), block b at [b][2 nf]
template <typename T>
__global__ void at_moments_kernel(const T *q, long long npts, int nf, double *part)
{
    __shared__ double red[256];
    for (int f = 0; f < nf; ++f) {
        for (int m = 0; m < 2; ++m) {
            double acc = 0.0;
            for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npts;
                 i += (long long)gridDim.x * blockDim.x) {
                const double v = (double)q[(size_t)f * npts + i];
                acc += m == 0 ? v : v * v;
            }
            red[threadIdx.x] = acc;
            __syncthreads();
            for (int o = blockDim.x / 2; o > 0; o >>= 1) {
                if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
                __syncthreads();
            }
            if (threadIdx.x == 0) part[(size_t)blockIdx.x * 2 * nf + 2 * f + m] = red[0];
            __syncthreads();
        }
    }
}

}  // namespace

extern "C" {

size_t at_system_workspace_bytes(const at_grid *grid, int64_t P, int L, int nfields)
{
    if (!grid || grid->dim != 3) { fail(AT_ERR_ARG, "the system needs dim = 3"); return 0; }
    if (nfields < 3 || nfields > 5) { fail(AT_ERR_ARG, "nfields must be 3, 4 or 5"); return 0; }
    Dims3 d;
    if (check_args3(grid, P, 2, L, &d) != AT_OK) return 0;
    const int w = grid->dtype == AT_F64 ? 8 : 4;
    return layout3(d, P, w, L, ring_slots(L, 2), nfields).total;
}

int at_create_system(const at_grid *grid, int64_t P, int L, int nfields, const double *kappa, double dt,
                     at_solver **out)
{
    g_err[0] = 0;
    if (!out) return fail(AT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || grid->dim != 3) return fail(AT_ERR_ARG, "the system needs dim = 3");
    if (nfields < 3 || nfields > 5) return fail(AT_ERR_ARG, "nfields must be 3, 4 or 5");
    if (!kappa) return fail(AT_ERR_ARG, "kappa is NULL");
    return create3d(grid, P, L, nfields, kappa, dt, out);
}

int at_moments(at_solver *h, double *out)
{
    g_err[0] = 0;
    if (!h || !out) return fail(AT_ERR_ARG, "NULL argument");
    if (h->dim != 3) return fail(AT_ERR_ARG, "at_moments is for 3D solvers");
    if (!h->has_state) return fail(AT_ERR_STATE, "at_moments before at_set_state");
    const long long npts = h->d3.n[0] * h->d3.n[1] * h->d3.n[2];
    const int blocks = (int)((npts + 255) / 256 < 4096 ? (npts + 255) / 256 : 4096);
    double *part = reinterpret_cast<double *>(h->ws + h->lay.bsub);
    cudaError_t e;
    if (h->w == 8) {
        at_moments_kernel<double><<<blocks, 256, 0, h->stream>>>(reinterpret_cast<const double *>(h->ws + h->lay.u),
                                                                 npts, h->nf, part);
    } else {
        at_moments_kernel<float><<<blocks, 256, 0, h->stream>>>(reinterpret_cast<const float *>(h->ws + h->lay.u),
                                                                npts, h->nf, part);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch at_moments_kernel");
    std::vector<double> host((size_t)blocks * 2 * h->nf);
    e = cudaMemcpyAsync(host.data(), part, host.size() * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(moments)");
    const int rc = read_status(h);
    if (rc != AT_OK) return rc;
    for (int f = 0; f < h->nf; ++f) {
        double s1 = 0.0, s2 = 0.0;
        for (int b = 0; b < blocks; ++b) {
            s1 += host[(size_t)b * 2 * h->nf + 2 * f];
            s2 += host[(size_t)b * 2 * h->nf + 2 * f + 1];
        }
        out[2 * f] = s1 / (double)npts;
        out[2 * f + 1] = s2 / (double)npts;
    }
    return AT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Arithmetic throughput probe (at_fma_peak): the measured FMA rate of this
// GPU for the roofline of ALU-bound variants (the FP64 state).
// ---------------------------------------------------------------------------
namespace {

static __device__ double g_probe_sink;

// kChains independent FMA chains per thread, kUnroll FMAs of each per trip:
// enough independent work to keep the FMA pipe of every SM issuing.
constexpr int kProbeChains = 8, kProbeUnroll = 8, kProbeThreads = 256, kProbeCtasPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) at_fma_probe(long long trips, T a, T b, double *sink)
{
    T x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (long long t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T acc = (T)0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc += x[c];
    if (acc == (T)-1.2345e30) *sink = (double)acc;   // never true; keeps the chains live
}

}  // namespace

extern "C" int at_fma_peak(int dtype, int64_t trips, double *fma_per_s)
{
    g_err[0] = 0;
    if (!fma_per_s) return fail(AT_ERR_ARG, "fma_per_s is NULL");
    if (dtype != AT_F64 && dtype != AT_F32) return fail(AT_ERR_ARG, "dtype must be AT_F64 or AT_F32");
    if (trips <= 0) return fail(AT_ERR_ARG, "trips must be positive");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    void *sink = nullptr;
    e = cudaGetSymbolAddress(&sink, g_probe_sink);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(probe sink)");
    cudaEvent_t ev[2];
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&ev[1])) != cudaSuccess) { cudaEventDestroy(ev[0]); return cuda_fail(e, "cudaEventCreate"); }
    const dim3 grid((unsigned)(sms * kProbeCtasPerSm)), block(kProbeThreads);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first launch warms up
        cudaEventRecord(ev[0], 0);
        if (dtype == AT_F64)
            at_fma_probe<double><<<grid, block>>>(trips, 0.9999999, 1e-7, static_cast<double *>(sink));
        else
            at_fma_probe<float><<<grid, block>>>(trips, 0.9999999f, 1e-7f, static_cast<double *>(sink));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return cuda_fail(e, "at_fma_probe");
    const double fmas = (double)grid.x * kProbeThreads * (double)trips * kProbeUnroll * kProbeChains;
    *fma_per_s = fmas / (ms * 1e-3);
    return AT_OK;
}
