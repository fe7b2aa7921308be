// esmm_api.cu -- grid/batch handles, launch domains, the SSP-RK3 step, CUDA
// graphs, the launch autotuner, and the C ABI declared in include/esmm.h.
//
// One right-hand-side evaluation (eqs. RMHDSemiU_O2p_ES / RMHDSemiJ_O2p_ES of
// Duan & Tang, arXiv 2107.12027, with B = 0) is four kinds of launch:
//   k_node   per padded node: primitive recovery, logs, metrics (ghost layers
//            applied by index mapping);
//   k_pairs  per direction: every two-point EC flux once;
//   k_iface  per direction: the ES interface flux;
//   k_update per node: flux differences, written out or fused with the
//            SSP-RK3 combination of the stage.
// A grid holds one problem or a batch of independent problems of different
// sizes in concatenated arrays; every kernel covers the whole batch in one
// launch through a block -> (problem, tile) map (esmm_device.cuh ProbArg).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <numeric>
#include <utility>
#include <vector>

#include "esmm.h"
#include "esmm_3d.h"
#include "esmm_device.cuh"
#include "esmm_kernels.cuh"
#include "esmm_launch.h"

using namespace esmm;

namespace {
// launch domains: which elements of each problem a kernel covers
// (D_TPAIR*, D_TIFACE*: the tiled launches of the RHD pair and interface
// kernels of the forward step, whose tile shape and persistence the tuner
// picks; the flat D_PAIR*, D_IFACE* serve the adjoint and RMHD kernels)
enum { D_PAD = 0, D_PAIR0, D_PAIR1, D_IFACE0, D_IFACE1, D_NODE, D_NODE2, D_MTILE, D_NEWTON,
       D_TPAIR0, D_TPAIR1, D_TIFACE0, D_TIFACE1, ND };
static_assert(ND + 4 == ESMM_TUNE_SLOTS, "esmm_tune reports every domain's block size and four tile shapes");
}  // namespace

struct esmm_grid {
    int dim;                         // 2, or 3 (then every call goes to g3)
    esmm3 *g3;
    int dev;
    int nprob;
    std::vector<ProbDesc> hpd;       // per-problem geometry and offsets
    std::vector<double> lo, hi;      // [nprob][2]
    ProbDesc *dpd;                   // device copy (batches)
    long long Ntot, Ptot;
    int phys;                        // ESMM_RHD or ESMM_RMHD
    int nv;                          // unknowns per node: 4 (RHD) or 8 (RMHD)
    double gamma;
    int p, w;
    esmm_params prm;
    cudaStream_t st;
    cudaStream_t own_st;             // stream created by the library (batches without one)
    int has_state;
    int xdot_zero;
    // state y^n = (cons, J, x), mesh velocity, stage buffers
    double *cons, *J, *x, *xdot;
    double *c1, *J1, *x1, *c2, *J2, *x2;
    // right-hand-side work arrays
    double *q;                       // [NQ][Ptot] (RMHD: [NQ_MHD][Ptot])
    double *cw;                      // [4][Ntot] Jacobi weights of the mesh iteration
    double *rs;                      // [2][Ntot] the iteration's residual on the displacement
    double *wr;                      // [6][Ntot] floats: weights and residual of the blocked sweeps
    float *q32;                      // [NQ32][Ptot] FP32 copies (RHD mixed form)
    double *inflow_dev;              // [8] primitive inflow state (ESMM_INFLOW ends)
    int needs_inflow, has_inflow;
    double *pg[3];                   // recovery warm starts (p; RMHD: Z), state -> stage 2 -> stage 3
    void *pairs;                     // [2][PMAX][4][Ptot] of the working precision (RHD)
    void *iflux;                     // [2][5][Ptot] (RMHD: [2][NF_MHD][Ptot]) of the working precision
    double *in_cons, *in_J, *in_x, *in_xdot, *out_dc, *out_dJ;  // host-mode staging
    // mesh redistribution
    double *grad, *om, *om2, *X, *Xn;
    unsigned long long *red;         // [nprob][NRED]
    double *dt_dev, *t_dev;          // [nprob]
    double *cflb;                    // [6][Ntot] the step solve: a_k, bmin_k, bmax_k per node
    double *npart;                   // [node-domain blocks][2][2] its per-block partial results
    DtSolve *ds;                     // [nprob] its state
    double *partials;                // totals: per-block partial sums
    double *tot_dev;                 // [nprob][3]
    int *status;                     // [0] failed recoveries, [1] bad initial states
    double *pin;                     // pinned host scalars [max(16, 3 nprob)]
    char msg[256];
    // launch domains: block size and tile order per kind (autotuned)
    int bs[ND];
    int order_lpt[ND];               // 1: largest problems first
    int tx[ND];                      // tile shape of the tiled flux launches (0: flat runs)
    int persist[ND];                 // 1: a persistent grid strides over the tiles
    int sms;                         // SMs of the grid's device
    int2 *tiles[ND];
    unsigned nblk[ND];
    size_t tiles_cap[ND];
    int doms_valid;
    // CUDA graph of one step (keyed by the dt argument, a parameter epoch and
    // the profiling mask it was captured with)
    cudaGraphExec_t graph;
    double graph_dt;
    int graph_epoch, epoch, graph_prof;
    int capturing;                   // this library is capturing the step graph
    int tuned;
    // profiling: launches per kind, CUDA events around the kinds in prof_mask
    int prof_mask;
    long long launches[ESMM_NKINDS];
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *ev;
    std::vector<cudaEvent_t> *pool;
    // event pairs recorded inside the step graph (re-recorded by every
    // replay), whether a replay's are still to be read, and the times and
    // counts read from replays so far
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *gev;
    int gev_pending;
    double gms[ESMM_NKINDS];
    long long gtimed[ESMM_NKINDS];
    // adjoint: per-step checkpoints [cons 4N | J N | x 2N | xdot 2N] and steps
    std::vector<double *> *ck;
    std::vector<double> *ck_dt;
    int ck_n;
    double *adjG, *adjGp;            // local Jacobian-vector contributions
    double *lam_a, *lam_b, *lam_c, *lam_v;
    // a slab of a decomposed grid (nslab > 0): its rows of the whole grid
    int nslab, slab;
    esmm_comm comm;
    int rows_g;                      // rows of the whole grid
    int own0, own1, ext0, ext1;      // own rows, held rows (global indices)
    int periodic1;                   // the whole grid is periodic in its second direction
    double per1;                     // that period
    double *xbuf;                    // pinned exchange buffers: send low/high, receive low/high
    size_t xbuf_n;                   // doubles per buffer
    double *vs_dev;                  // [2][2] a slab's Newton values and slopes
    const void *mesh_disp;           // the displacement x^[mu] - x^n of the last mesh step
};

namespace {

constexpr int BS = 256;

inline unsigned nblk(long long n, int bs = BS) { return (unsigned)((n + bs - 1) / bs); }

cudaEvent_t pool_get(esmm_grid *g)
{
    if (!g->pool->empty()) {
        cudaEvent_t e = g->pool->back();
        g->pool->pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Counts one launch of a kind and, when the kind is profiled (and the stream
// is not being captured), brackets it with CUDA events on the grid's stream.
struct Prof {
    esmm_grid *g;
    int kind;
    cudaEvent_t a = nullptr;
    bool in_graph = false;
    Prof(esmm_grid *g_, int kind_) : g(g_), kind(kind_)
    {
        g->launches[kind] += 1;
        if (!(g->prof_mask & (1 << kind))) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(g->st, &cs);
        if (cs == cudaStreamCaptureStatusNone) {
            a = pool_get(g);
            cudaEventRecord(a, g->st);
        } else if (g->capturing) {   // inside the library's own step graph: an event node
            a = pool_get(g);
            in_graph = true;
            cudaEventRecordWithFlags(a, g->st, cudaEventRecordExternal);
        }
    }
    ~Prof()
    {
        if (!a) return;
        cudaEvent_t b = pool_get(g);
        if (in_graph) {
            cudaEventRecordWithFlags(b, g->st, cudaEventRecordExternal);
            g->gev[kind].push_back({a, b});
        } else {
            cudaEventRecord(b, g->st);
            g->ev[kind].push_back({a, b});
        }
    }
};

int fail(esmm_grid *g, int code, const char *what, cudaError_t e = cudaSuccess)
{
    if (g) {
        if (e != cudaSuccess) snprintf(g->msg, sizeof g->msg, "%s: %s", what, cudaGetErrorString(e));
        else snprintf(g->msg, sizeof g->msg, "%s", what);
    }
    return code;
}

#define CK(call)                                                         \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return fail(g, ESMM_ERR_CUDA, #call, e_); \
    } while (0)

Phys phys(const esmm_grid *g)
{
    Phys ph;
    ph.gamma = g->gamma;
    ph.eps = g->prm.weno_eps;
    // FP64: switch to the series below 1e-4 (its dropped term is < 1e-17);
    // FP32 bulk: below 1e-2, where the FP32 quotient would lose ~6 digits.
    ph.ln_thr = g->prm.precision == ESMM_MIXED ? 1.0e-2 : 1.0e-4;
    ph.gm1i = 1.0 / (g->gamma - 1.0);
    // sign switch: rounding noise of the projected jump (FP64 / FP32 bulk)
    ph.sign_tol = g->prm.precision == ESMM_MIXED ? 1.0e-5 : 1.0e-10;
    double a[3][3] = {{1.0, 0.0, 0.0}, {4.0 / 3.0, -1.0 / 6.0, 0.0}, {1.5, -0.3, 1.0 / 30.0}};
    for (int n = 0; n < PMAX; ++n) ph.alpha[n] = a[g->p - 1][n];
    ph.p = g->p;
    ph.w = g->w;
    return ph;
}

long long dom_count(const Geom &G, int kind, int p)
{
    switch (kind) {
    case D_PAD: return G.P;
    case D_PAIR0: case D_TPAIR0: return (long long)(G.nx + p) * G.ny;
    case D_PAIR1: case D_TPAIR1: return (long long)(G.ny + p) * G.nx;
    case D_IFACE0: case D_TIFACE0: return (long long)(G.nx + 1) * G.ny;
    case D_IFACE1: case D_TIFACE1: return (long long)(G.ny + 1) * G.nx;
    case D_NODE: return G.N;
    case D_MTILE:   // one block of MT_THREADS per MT_TX x MT_TY tile
        return (long long)((G.nx + MT_TX - 1) / MT_TX) * ((G.ny + MT_TY - 1) / MT_TY) * MT_THREADS;
    case D_NEWTON:  // DT_NPT nodes per thread
        return (G.N + DT_NPT - 1) / DT_NPT;
    default: return 2 * G.N;
    }
}

// tiles (blocks) of one problem in a domain: flat runs of bs sites, or, for
// a tiled flux launch with tx > 0, tx x (bs / tx) tiles of the sweep's sites
long long dom_blocks(const esmm_grid *g, const Geom &G, int kind)
{
    const int bs = g->bs[kind], tx = g->tx[kind];
    if (tx < 0 && (kind == D_TIFACE0 || kind == D_TIFACE1))   // the fused sweep: bs / 32 lines per tile
        return sweep_tiles(G, kind == D_TIFACE1 ? 1 : 0, g->p, bs / 32);
    if (tx > 0 && kind >= D_TPAIR0 && kind <= D_TIFACE1) {
        const int dir = (kind == D_TPAIR1 || kind == D_TIFACE1) ? 1 : 0;
        const int ext = kind <= D_TPAIR1 ? g->p : 1;
        const long long nd = dir == 0 ? G.nx : G.ny, no = dir == 0 ? G.ny : G.nx;
        const long long Ei = dir == 0 ? nd + ext : no, Ej = dir == 0 ? no : nd + ext, ty = bs / tx;
        return ((Ei + tx - 1) / tx) * ((Ej + ty - 1) / ty);
    }
    return (long long)nblk(dom_count(G, kind, g->p), bs);
}

// The 2D RHD flux variant of both sweep directions (esmm_params.sweep):
// the fused kernel (tx = -1 in the interface domains, 128 threads = 4 lines
// per block) or the pair and interface kernels (flat runs of 128 sites);
// ESMM_SWEEP_AUTO starts from the fused kernel until the tuner decides.
void set_sweep(esmm_grid *g, int sweep)
{
    for (int k : {D_TPAIR0, D_TPAIR1, D_TIFACE0, D_TIFACE1}) {
        g->bs[k] = 128;
        g->tx[k] = 0;
        g->persist[k] = 0;
    }
    if (sweep != ESMM_SWEEP_SPLIT) g->tx[D_TIFACE0] = g->tx[D_TIFACE1] = -1;
    g->doms_valid = 0;
}

// (Re)build the block -> (problem, tile) map of one kind.
int build_dom(esmm_grid *g, int kind)
{
    if (g->nprob == 1) {
        g->nblk[kind] = (unsigned)dom_blocks(g, g->hpd[0].g, kind);
        return ESMM_OK;
    }
    std::vector<int> order(g->nprob);
    std::iota(order.begin(), order.end(), 0);
    if (g->order_lpt[kind])
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return dom_blocks(g, g->hpd[a].g, kind) > dom_blocks(g, g->hpd[b].g, kind);
        });
    std::vector<int2> map;
    for (int b : order) {
        long long nb = dom_blocks(g, g->hpd[b].g, kind);
        for (long long k = 0; k < nb; ++k) map.push_back(make_int2(b, (int)k));
    }
    if (map.size() > g->tiles_cap[kind]) {
        if (g->tiles[kind]) cudaFree(g->tiles[kind]);
        g->tiles[kind] = nullptr;
        CK(cudaMalloc((void **)&g->tiles[kind], map.size() * sizeof(int2)));
        g->tiles_cap[kind] = map.size();
    }
    CK(cudaMemcpyAsync(g->tiles[kind], map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice, g->st));
    CK(cudaStreamSynchronize(g->st));
    g->nblk[kind] = (unsigned)map.size();
    return ESMM_OK;
}

int ensure_doms(esmm_grid *g)
{
    if (g->needs_inflow && !g->has_inflow) return fail(g, ESMM_ERR_STATE, "an inflow end without an inflow state");
    if (g->doms_valid) return ESMM_OK;
    for (int k = 0; k < ND; ++k) {
        int rc = build_dom(g, k);
        if (rc) return rc;
    }
    g->doms_valid = 1;
    return ESMM_OK;
}

LaunchDom dom(const esmm_grid *g, int kind)
{
    LaunchDom L;
    L.pa.pd = g->nprob == 1 ? nullptr : g->dpd;
    L.pa.tiles = g->nprob == 1 ? nullptr : g->tiles[kind];
    L.pa.one = g->hpd[0];
    L.nblk = g->nblk[kind];
    L.bs = g->bs[kind];
    if (kind >= D_TPAIR0 && kind <= D_TIFACE1) {
        L.tx = g->tx[kind];
        L.ntiles = g->nblk[kind];
        if (g->persist[kind]) {   // as many blocks as the SMs hold at once
            const int k = kind <= D_TPAIR1 ? 0 : 1;
            const bool f32 = g->prm.precision == ESMM_MIXED;
            const int per_sm = L.tx < 0 ? (f32 ? sweep_occupancy_f32(g->p, g->w, L.bs)
                                               : sweep_occupancy_f64(g->p, g->w, L.bs))
                                        : (f32 ? flux_occupancy_f32(k, g->p, g->w, L.bs)
                                               : flux_occupancy_f64(k, g->p, g->w, L.bs));
            L.nblk = (unsigned)std::min<long long>(L.ntiles, (long long)per_sm * g->sms);
        }
    }
    return L;
}

// a one-problem domain for problem b with block size bs (state set-up/read-out)
LaunchDom dom_one(const esmm_grid *g, int b, int kind, int bs = BS)
{
    LaunchDom L;
    L.pa.pd = nullptr;
    L.pa.tiles = nullptr;
    L.pa.one = g->hpd[b];
    L.nblk = nblk(dom_count(g->hpd[b].g, kind, g->p), bs);
    L.bs = bs;
    return L;
}

// the FP32 copies of the node arrays, written and read in the RHD mixed form
float *q32_of(const esmm_grid *g)
{
    return g->phys == ESMM_RHD && g->prm.precision == ESMM_MIXED ? g->q32 : nullptr;
}

void launch_node(const esmm_grid *g, const LaunchDom &L, const double *cons, const double *J, const double *x,
                 const double *xdot, const double *pg_in, double *pg_out, double *q, bool exact_logs)
{
    float *q32 = q32_of(g);
    const double *in = g->has_inflow ? g->inflow_dev : nullptr;
    const int f32_logs = q32 && !exact_logs;
    const double gg = (g->gamma - 1.0) / g->gamma;
    if (g->p == 1)
        k_node<1><<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->gamma, gg, cons, J, x, xdot, pg_in, pg_out, q, g->status,
                                              q32, in, f32_logs);
    else if (g->p == 2)
        k_node<2><<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->gamma, gg, cons, J, x, xdot, pg_in, pg_out, q, g->status,
                                              q32, in, f32_logs);
    else
        k_node<3><<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->gamma, gg, cons, J, x, xdot, pg_in, pg_out, q, g->status,
                                              q32, in, f32_logs);
}

// the node pass; exact_logs: FP64 logarithms in every form (the totals)
void node(esmm_grid *g, const double *cons, const double *J, const double *x, const double *xdot,
          const double *pg_in, double *pg_out, bool exact_logs = false)
{
    Prof pr_(g, ESMM_KIND_NODE);
    if (g->phys == ESMM_RMHD)
        launch_node_mhd(dom(g, D_PAD), g->p, g->gamma, cons, J, x, xdot, pg_in, pg_out, g->q, g->status,
                        g->has_inflow ? g->inflow_dev : nullptr,
                        g->prm.precision == ESMM_MIXED && !exact_logs, g->st);
    else
        launch_node(g, dom(g, D_PAD), cons, J, x, xdot, pg_in, pg_out, g->q, exact_logs);
}

// both sweeps of the flux kernels for the node data in g->q
void fluxes(esmm_grid *g)
{
    Phys ph = phys(g);
    bool f32 = g->prm.precision == ESMM_MIXED;
    for (int dir = 0; dir < 2; ++dir) {
        const bool rmhd = g->phys == ESMM_RMHD;
        LaunchDom Lp = dom(g, dir == 0 ? D_TPAIR0 : D_TPAIR1);
        LaunchDom Li = dom(g, rmhd ? (dir == 0 ? D_IFACE0 : D_IFACE1) : (dir == 0 ? D_TIFACE0 : D_TIFACE1));
        if (rmhd) {   // two-point fluxes summed inside the interface kernel
            Prof pr_(g, ESMM_KIND_IFACE);
            if (f32) launch_iface_mhd_f32(Li, ph, g->q, g->iflux, dir, g->st);
            else launch_iface_mhd(Li, ph, g->q, g->iflux, dir, g->st);
            continue;
        }
        if (Li.tx < 0) {   // the fused sweep: pair fluxes kept in shared memory
            Prof pr_(g, ESMM_KIND_IFACE);
            if (f32) launch_sweep_f32(Li, ph, g->q, g->q32, g->iflux, dir, g->st);
            else launch_sweep_f64(Li, ph, g->q, nullptr, g->iflux, dir, g->st);
            continue;
        }
        {
            Prof pr_(g, ESMM_KIND_PAIRS);
            if (f32) launch_pairs_f32(Lp, ph, g->q, g->q32, g->pairs, dir, g->st);
            else launch_pairs_f64(Lp, ph, g->q, nullptr, g->pairs, dir, g->st);
        }
        {
            Prof pr_(g, ESMM_KIND_IFACE);
            if (f32) launch_iface_f32(Li, ph, g->q, g->q32, g->pairs, g->iflux, dir, g->st);
            else launch_iface_f64(Li, ph, g->q, nullptr, g->pairs, g->iflux, dir, g->st);
        }
    }
}

void update(esmm_grid *g, double *dcons, double *dJ, const double *cn, const double *Jn, const double *xn,
            const double *cs, const double *Js, const double *xs, const double *xdot, double A, double B,
            double *co, double *Jo, double *xo)
{
    Prof pr_(g, ESMM_KIND_UPDATE);
    LaunchDom L = dom(g, D_NODE);
    if (g->phys == ESMM_RMHD && g->prm.precision == ESMM_MIXED)
        launch_update_mhd_f32(L, g->q, g->iflux, dcons, dJ, cn, Jn, xn, cs, Js, xs, xdot, A, B, g->dt_dev, co, Jo,
                              xo, g->st);
    else if (g->phys == ESMM_RMHD)
        launch_update_mhd(L, g->q, g->iflux, dcons, dJ, cn, Jn, xn, cs, Js, xs, xdot, A, B, g->dt_dev, co, Jo, xo,
                          g->st);
    else if (g->prm.precision == ESMM_MIXED)
        k_update<float><<<L.nblk, L.bs, 0, g->st>>>(L.pa, (const float *)g->iflux, dcons, dJ, cn, Jn, xn, cs, Js, xs,
                                                    xdot, A, B, g->dt_dev, co, Jo, xo);
    else
        k_update<double><<<L.nblk, L.bs, 0, g->st>>>(L.pa, (const double *)g->iflux, dcons, dJ, cn, Jn, xn, cs, Js,
                                                     xs, xdot, A, B, g->dt_dev, co, Jo, xo);
}

unsigned nprob_blocks(const esmm_grid *g) { return nblk(g->nprob, 128); }

// static spectral radius of the state (when dt is to come from eq. cfl);
// requires g->q of the state with a static mesh and the slots reset.  With a
// moving mesh the speed bounds of every node go to g->cflb for the step solve.
void step_radius(esmm_grid *g, double dt, bool moving)
{
    if (dt > 0.0) return;
    Prof pr_(g, ESMM_KIND_OTHER);
    LaunchDom L = dom(g, D_NODE);
    double *cflb = moving ? g->cflb : nullptr;
    if (g->phys == ESMM_RMHD)   // at most 256 threads per block, whatever the node kind's tuned size: the
                                // eigen-system holds up to 255 registers per thread (RMHD grids are single
                                // problems)
        launch_cfl_mhd(dom_one(g, 0, D_NODE, std::min(L.bs, 256)), g->gamma, g->q, g->J, g->red,
                       g->prm.precision == ESMM_MIXED, cflb, g->st);
    else
        k_cfl<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->gamma, g->gamma / (g->gamma - 1.0), g->q, g->J, g->red,
                                          q32_of(g), cflb);
}

// the step into dt_dev (and the limiter, scaled where the displacement alone
// breaks eq. cfl, into slot 1), after the radius and (when the mesh moves) the
// mesh chain up to k_mesh_tau: the set-up, then, for a CFL step with mesh
// motion, the DT_NEWTON evaluations of the solve (each a no-op once a
// problem's solve has ended; a fixed count keeps the step graph-capturable)
void step_dt(esmm_grid *g, double dt, bool moving)
{
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_dt<<<nprob_blocks(g), 128, 0, g->st>>>(g->nprob, g->prm.cfl, dt, g->red, g->ds, g->dt_dev);
    }
    if (dt > 0.0 || !moving) return;
    LaunchDom L = dom(g, D_NEWTON);
    for (int it = 0; it < DT_NEWTON; ++it) {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_dt_newton<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->prm.cfl, g->cflb, g->red, g->ds, g->npart, g->dt_dev,
                                                nullptr);
    }
}

void red_init(esmm_grid *g)
{
    Prof pr_(g, ESMM_KIND_OTHER);
    k_red_init<<<nprob_blocks(g), 128, 0, g->st>>>(g->nprob, g->red);
}

// sweeps per launch of k_mesh_sweeps in the mixed form (FP32: all ten sweeps
// of the default in one launch); the FP64 form sweeps once per launch
// (k_mesh_sweep), since the blocked kernel's halo work costs FP64 issue slots
constexpr int MT_SB32 = 10;

// The Jacobi sweeps (k_mesh_sweeps) and the limiter, in working type T (the
// weights are in g->cw; the blocked sweeps read them, with the residual, in
// T from g->wr); the displacement is left at g->mesh_disp.
template <typename T, int SB>
int mesh_sweeps_tau(esmm_grid *g, const LaunchDom &L)
{
    T *bufs[2] = {reinterpret_cast<T *>(g->X), reinterpret_cast<T *>(g->Xn)};
    const T *Dd = bufs[0];
    if (g->prm.mu == 0) {
        CK(cudaMemsetAsync(bufs[0], 0, sizeof(T) * 2 * g->Ntot, g->st));
    } else if constexpr (SB == 1) {   // FP64: one sweep per launch
        {
            Prof pr_(g, ESMM_KIND_MESH);
            k_mesh_resid<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->x, g->cw, g->rs);
        }
        const double *in = nullptr;
        int b = 0;
        for (int nu = 0; nu < g->prm.mu; ++nu) {
            Prof pr_(g, ESMM_KIND_MESH);
            double *out = reinterpret_cast<double *>(bufs[b]);
            k_mesh_sweep<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->cw, g->rs, in, out);
            in = out;
            b ^= 1;
        }
        Dd = reinterpret_cast<const T *>(in);
    } else {
        LaunchDom Lt = dom(g, D_MTILE);
        T *wr = reinterpret_cast<T *>(g->wr);
        {
            Prof pr_(g, ESMM_KIND_MESH);
            k_mesh_wr<T><<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->x, g->cw, wr);
        }
        const T *in = nullptr;
        int b = 0;
        for (int done = 0; done < g->prm.mu; done += SB) {
            Prof pr_(g, ESMM_KIND_MESH);
            k_mesh_sweeps<T, SB><<<Lt.nblk, MT_THREADS, mesh_sweeps_smem<T, SB>(), g->st>>>(
                Lt.pa, wr, in, bufs[b], std::min(SB, g->prm.mu - done));
            in = bufs[b];
            b ^= 1;
        }
        Dd = in;
    }
    {
        Prof pr_(g, ESMM_KIND_MESH);
        k_mesh_tau<T><<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->x, Dd, g->q, g->J, g->red, g->cflb);
    }
    g->mesh_disp = Dd;
    return ESMM_OK;
}

// ... then the step (step_dt) and the mesh velocity from the displacement
template <typename T, int SB>
int mesh_finish(esmm_grid *g, double dt, const LaunchDom &L, const LaunchDom &L2)
{
    int rc = mesh_sweeps_tau<T, SB>(g, L);
    if (rc) return rc;
    step_dt(g, dt, true);
    {
        Prof pr_(g, ESMM_KIND_MESH);
        k_mesh_xdot<T><<<L2.nblk, L2.bs, 0, g->st>>>(L2.pa, (const T *)g->mesh_disp, g->red, g->dt_dev, g->xdot);
    }
    return ESMM_OK;
}

// the shared-memory limit of the sweep kernels (once per process and device
// is enough; cheap to repeat)
int mesh_sweeps_init(esmm_grid *g)
{
    CK(cudaFuncSetAttribute(k_mesh_sweeps<float, MT_SB32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)mesh_sweeps_smem<float, MT_SB32>()));
    return ESMM_OK;
}

// The step: mesh target and limiter (when the mesh moves), dt (k_dt) and the
// mesh velocity into g->xdot.  Requires g->q of the state, the slots reset
// and the radius (step_radius) when dt <= 0.
int mesh_core(esmm_grid *g, double dt)
{
    if (!g->prm.move_mesh) {
        step_dt(g, dt, false);
        if (!g->xdot_zero) {
            CK(cudaMemsetAsync(g->xdot, 0, sizeof(double) * 2 * g->Ntot, g->st));
            g->xdot_zero = 1;
        }
        return ESMM_OK;
    }
    g->xdot_zero = 0;
    LaunchDom L = dom(g, D_NODE), L2 = dom(g, D_NODE2);
    {
        Prof pr_(g, ESMM_KIND_MESH);
        // the Laplacian goes to om2, which the filter overwrites only after k_mesh_omega
        k_mesh_grad<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->prm.monitor == ESMM_MONITOR_LNRHO, g->prm.alpha_lap > 0.0,
                                                g->q, g->grad, g->om2, g->red);
    }
    {
        Prof pr_(g, ESMM_KIND_MESH);
        k_mesh_omega<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->prm.alpha, g->prm.alpha_lap, g->grad, g->om2, g->red,
                                                 g->om);
    }
    double *om = g->om, *om2 = g->om2;
    for (int f = 0; f < g->prm.n_filter; ++f) {
        Prof pr_(g, ESMM_KIND_MESH);
        k_mesh_filter<<<L.nblk, L.bs, 0, g->st>>>(L.pa, om, om2);
        std::swap(om, om2);
    }
    if (g->prm.mu > 0) {
        Prof pr_(g, ESMM_KIND_MESH);
        k_mesh_weights<<<L.nblk, L.bs, 0, g->st>>>(L.pa, om, g->cw);
    }
    // the mu sweeps on the displacement, SB per launch (FP32 in the mixed form)
    if (g->prm.precision == ESMM_MIXED) return mesh_finish<float, MT_SB32>(g, dt, L, L2);
    return mesh_finish<double, 1>(g, dt, L, L2);
}

int stages(esmm_grid *g);

// One step of every problem (asynchronous on the grid's stream).
int rk_step_async(esmm_grid *g, double dt)
{
    int rc;
    if ((rc = ensure_doms(g))) return rc;
    // the state's node data with a static mesh: CFL step and monitor (Sec. 5)
    node(g, g->cons, g->J, g->x, nullptr, g->pg[0], g->pg[1]);
    red_init(g);
    step_radius(g, dt, g->prm.move_mesh);
    if ((rc = mesh_core(g, dt))) return rc;
    // stage 1: y1 = y^n + dt L(y^n); only the temporal metrics change
    {
        Prof pr_(g, ESMM_KIND_NODE);
        LaunchDom L = dom(g, D_PAD);
        k_tmetric<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->xdot, g->q, q32_of(g));
    }
    return stages(g);
}

// The three SSP-RK3 stages, the node data of the state (with the step's mesh
// velocity) already in g->q and the step in dt_dev.
int stages(esmm_grid *g)
{
    fluxes(g);
    update(g, nullptr, nullptr, g->cons, g->J, g->x, g->cons, g->J, g->x, g->xdot, 0.0, 1.0, g->c1, g->J1, g->x1);
    // stage 2: y2 = 3/4 y^n + 1/4 (y1 + dt L(y1))
    node(g, g->c1, g->J1, g->x1, g->xdot, g->pg[1], g->pg[2]);
    fluxes(g);
    update(g, nullptr, nullptr, g->cons, g->J, g->x, g->c1, g->J1, g->x1, g->xdot, 0.75, 0.25, g->c2, g->J2, g->x2);
    // stage 3: y^{n+1} = 1/3 y^n + 2/3 (y2 + dt L(y2)), in place
    node(g, g->c2, g->J2, g->x2, g->xdot, g->pg[2], g->pg[0]);
    fluxes(g);
    update(g, nullptr, nullptr, g->cons, g->J, g->x, g->c2, g->J2, g->x2, g->xdot, 1.0 / 3.0, 2.0 / 3.0, g->cons,
           g->J, g->x);
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_time<<<nprob_blocks(g), 128, 0, g->st>>>(g->nprob, g->dt_dev, g->t_dev);
    }
    CK(cudaGetLastError());
    return ESMM_OK;
}

int check_c2p(esmm_grid *g)
{
    int h[2];
    CK(cudaMemcpyAsync(h, g->status, sizeof h, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    if (h[0] > 0) {
        CK(cudaMemsetAsync(g->status, 0, sizeof(int), g->st));
        snprintf(g->msg, sizeof g->msg, "primitive recovery failed at %d node(s)", h[0]);
        return ESMM_ERR_C2P;
    }
    return ESMM_OK;
}

void drop_graph(esmm_grid *g)
{
    if (g->graph) {
        // a replay may still be recording the graph's events
        cudaStreamSynchronize(g->st);
        cudaGraphExecDestroy(g->graph);
    }
    g->graph = nullptr;
    if (g->gev)
        for (int k = 0; k < ESMM_NKINDS; ++k) {
            for (auto &pr : g->gev[k]) { g->pool->push_back(pr.first); g->pool->push_back(pr.second); }
            g->gev[k].clear();
        }
    g->gev_pending = 0;
}

// Add the device times of the last replay's graph events to the profile
// (before the next replay records them again).
int collect_graph_prof(esmm_grid *g)
{
    if (!g->gev_pending) return ESMM_OK;
    for (int k = 0; k < ESMM_NKINDS; ++k)
        for (auto &pr : g->gev[k]) {
            float t = 0.0f;
            CK(cudaEventSynchronize(pr.second));
            CK(cudaEventElapsedTime(&t, pr.first, pr.second));
            g->gms[k] += t;
            g->gtimed[k] += 1;
        }
    g->gev_pending = 0;
    return ESMM_OK;
}

void free_all(esmm_grid *g)
{
    double **bufs[] = {&g->cons, &g->J, &g->x, &g->xdot, &g->c1, &g->J1, &g->x1, &g->c2, &g->J2, &g->x2,
                       &g->q, &g->pg[0], &g->pg[1], &g->pg[2], &g->in_cons, &g->in_J, &g->in_x, &g->in_xdot,
                       &g->out_dc, &g->out_dJ, &g->grad, &g->om, &g->om2, &g->cw, &g->rs, &g->wr, &g->X, &g->Xn,
                       &g->dt_dev,
                       &g->t_dev, &g->partials, &g->tot_dev, &g->inflow_dev, &g->cflb, &g->npart, &g->vs_dev};
    for (double **b : bufs)
        if (*b) { cudaFree(*b); *b = nullptr; }
    drop_graph(g);
    if (g->pairs) cudaFree(g->pairs);
    if (g->q32) cudaFree(g->q32);
    g->q32 = nullptr;
    if (g->iflux) cudaFree(g->iflux);
    if (g->red) cudaFree(g->red);
    if (g->ds) cudaFree(g->ds);
    g->ds = nullptr;
    if (g->status) cudaFree(g->status);
    if (g->dpd) cudaFree(g->dpd);
    if (g->pin) cudaFreeHost(g->pin);
    if (g->xbuf) cudaFreeHost(g->xbuf);
    g->xbuf = nullptr;
    for (int k = 0; k < ND; ++k)
        if (g->tiles[k]) { cudaFree(g->tiles[k]); g->tiles[k] = nullptr; }
    if (g->ev) {
        for (int k = 0; k < ESMM_NKINDS; ++k)
            for (auto &pr : g->ev[k]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
        delete[] g->ev;
        g->ev = nullptr;
    }
    if (g->gev) {   // drop_graph above returned them to the pool
        delete[] g->gev;
        g->gev = nullptr;
    }
    if (g->pool) {
        for (cudaEvent_t e : *g->pool) cudaEventDestroy(e);
        delete g->pool;
        g->pool = nullptr;
    }
    if (g->ck) {
        for (double *b : *g->ck) cudaFree(b);
        delete g->ck;
        g->ck = nullptr;
    }
    if (g->ck_dt) { delete g->ck_dt; g->ck_dt = nullptr; }
    double **abufs[] = {&g->adjG, &g->adjGp, &g->lam_a, &g->lam_b, &g->lam_c, &g->lam_v};
    for (double **b : abufs)
        if (*b) { cudaFree(*b); *b = nullptr; }
    if (g->own_st) { cudaStreamDestroy(g->own_st); g->own_st = nullptr; }
    g->pairs = g->iflux = nullptr;
    g->red = nullptr;
    g->status = nullptr;
    g->dpd = nullptr;
    g->pin = nullptr;
}

int copy_in(esmm_grid *g, double *dst, const double *src, size_t n, int mem)
{
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double),
                       mem == ESMM_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->st));
    return ESMM_OK;
}

int copy_out(esmm_grid *g, double *dst, const double *src, size_t n, int mem)
{
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double),
                       mem == ESMM_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->st));
    return ESMM_OK;
}

void release(esmm_grid *g)
{
    if (g->g3) esmm3_destroy(g->g3);
    g->g3 = nullptr;
    free_all(g);
    delete g;   // destroys the member vectors
}

// a dim = 3 grid: a shell that forwards to the 3D handle
int create3(esmm_grid **out, const int n[3], const double lo[3], const double hi[3], const int bc[3], void *stream)
{
    *out = nullptr;
    esmm_grid *g = new (std::nothrow) esmm_grid;
    if (!g) return ESMM_ERR_ARG;
    memset((void *)g, 0, sizeof *g);
    for (int d = 0; d < 3; ++d)
        if (bc[d] == ESMM_INFLOW) g->needs_inflow = 1;
    new (&g->hpd) std::vector<ProbDesc>();
    new (&g->lo) std::vector<double>();
    new (&g->hi) std::vector<double>();
    g->dim = 3;
    g->nprob = 1;
    g->phys = ESMM_RMHD;
    g->nv = 8;
    int rc = esmm3_create(&g->g3, n, lo, hi, bc, stream);
    if (rc) {
        delete g;
        return rc;
    }
    *out = g;
    return ESMM_OK;
}

// Create a grid of nprob problems: n, lo, hi, bc are [nprob][2].
int create(esmm_grid **out, int nprob, const int *n, const double *lo, const double *hi, const int *bc,
           int phys, void *stream, bool own_stream)
{
    *out = nullptr;
    esmm_grid *g = new (std::nothrow) esmm_grid;
    if (!g) return ESMM_ERR_ARG;
    {
        // zero every plain member, then re-construct the vectors in place
        memset((void *)g, 0, sizeof *g);
        new (&g->hpd) std::vector<ProbDesc>();
        new (&g->lo) std::vector<double>();
        new (&g->hi) std::vector<double>();
    }
    g->dim = 2;
    g->ev = new (std::nothrow) std::vector<std::pair<cudaEvent_t, cudaEvent_t>>[ESMM_NKINDS];
    g->gev = new (std::nothrow) std::vector<std::pair<cudaEvent_t, cudaEvent_t>>[ESMM_NKINDS];
    g->pool = new (std::nothrow) std::vector<cudaEvent_t>;
    g->ck = new (std::nothrow) std::vector<double *>;
    g->ck_dt = new (std::nothrow) std::vector<double>;
    if (!g->ev || !g->gev || !g->pool || !g->ck || !g->ck_dt || cudaGetDevice(&g->dev) != cudaSuccess) {
        release(g);
        return ESMM_ERR_CUDA;
    }
    g->nprob = nprob;
    g->st = (cudaStream_t)stream;
    if (!stream && own_stream) {
        if (cudaStreamCreateWithFlags(&g->own_st, cudaStreamNonBlocking) != cudaSuccess) {
            release(g);
            return ESMM_ERR_CUDA;
        }
        g->st = g->own_st;
    }
    long long on = 0, op = 0;
    for (int b = 0; b < nprob; ++b) {
        ProbDesc D;
        Geom &G = D.g;
        G.nx = n[2 * b];
        G.ny = n[2 * b + 1];
        G.px = G.nx + 2 * GH;
        G.py = G.ny + 2 * GH;
        G.P = (long long)G.px * G.py;
        G.N = (long long)G.nx * G.ny;
        G.bc0 = bc[2 * b];
        G.bc1 = bc[2 * b + 1];
        G.own0 = 0;
        G.own1 = G.ny;
        if (G.bc0 == ESMM_INFLOW || G.bc1 == ESMM_INFLOW) g->needs_inflow = 1;
        G.per0 = hi[2 * b] - lo[2 * b];
        G.per1 = hi[2 * b + 1] - lo[2 * b + 1];
        D.on = on;
        D.op = op;
        on += G.N;
        op += G.P;
        g->hpd.push_back(D);
        for (int k = 0; k < 2; ++k) { g->lo.push_back(lo[2 * b + k]); g->hi.push_back(hi[2 * b + k]); }
    }
    g->Ntot = on;
    g->Ptot = op;
    g->phys = phys;
    g->nv = phys == ESMM_RMHD ? 8 : 4;
    g->gamma = 5.0 / 3.0;
    g->p = 2;
    g->w = 5;
    g->prm.cfl = 0.4;
    g->prm.weno_eps = 1e-6;
    g->prm.monitor = ESMM_MONITOR_LNRHO;
    g->prm.alpha = 20.0;
    g->prm.n_filter = 4;
    g->prm.alpha_lap = 0.0;
    g->prm.sweep = ESMM_SWEEP_AUTO;
    g->prm.mu = 10;
    g->prm.move_mesh = 1;
    g->prm.precision = ESMM_FP64;
    for (int k = 0; k < ND; ++k) {
        g->bs[k] = ((k >= D_PAIR0 && k <= D_IFACE1) || k >= D_TPAIR0) ? 128 : BS;
        g->tx[k] = 0;
        g->persist[k] = 0;
    }
    set_sweep(g, ESMM_SWEEP_AUTO);
    if (cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->dev) != cudaSuccess || g->sms < 1)
        g->sms = 1;

    size_t N = (size_t)g->Ntot, P = (size_t)g->Ptot, d = sizeof(double), nv = (size_t)g->nv;
    size_t nb_max = (size_t)(N / 64 + (size_t)nprob + 64);   // node-domain blocks at >= 64 threads
    size_t nq = phys == ESMM_RMHD ? (size_t)NQ_MHD : (size_t)NQ;
    struct { double **p; size_t n; } al[] = {
        {&g->cons, nv * N}, {&g->J, N}, {&g->x, 2 * N}, {&g->xdot, 2 * N}, {&g->c1, nv * N}, {&g->J1, N},
        {&g->x1, 2 * N}, {&g->c2, nv * N}, {&g->J2, N}, {&g->x2, 2 * N}, {&g->q, nq * P},
        {&g->pg[0], N}, {&g->pg[1], N}, {&g->pg[2], N}, {&g->out_dc, nv * N}, {&g->out_dJ, N},
        {&g->grad, N}, {&g->om, N}, {&g->om2, N}, {&g->cw, 4 * N}, {&g->rs, 2 * N}, {&g->wr, 3 * N}, {&g->X, 2 * N},
        {&g->Xn, 2 * N},
        {&g->dt_dev, (size_t)nprob}, {&g->t_dev, (size_t)nprob}, {&g->partials, 3 * nb_max}, {&g->inflow_dev, 8},
        {&g->cflb, 6 * N}, {&g->npart, 4 * nb_max},
        {&g->tot_dev, 3 * (size_t)nprob}};
    for (auto &a : al)
        if (cudaMalloc((void **)a.p, a.n * d) != cudaSuccess) { release(g); return ESMM_ERR_CUDA; }
    if (nprob == 1) {   // host-pointer staging of esmm_rhs (single problems only)
        if (cudaMalloc((void **)&g->in_cons, nv * N * d) != cudaSuccess ||
            cudaMalloc((void **)&g->in_J, N * d) != cudaSuccess ||
            cudaMalloc((void **)&g->in_x, 2 * N * d) != cudaSuccess ||
            cudaMalloc((void **)&g->in_xdot, 2 * N * d) != cudaSuccess) {
            release(g);
            return ESMM_ERR_CUDA;
        }
    }
    size_t npairs = phys == ESMM_RMHD ? 1 : (size_t)2 * PMAX * 4 * P;
    size_t nflux = phys == ESMM_RMHD ? (size_t)2 * NF_MHD * P : (size_t)2 * 5 * P;
    if ((phys == ESMM_RHD && cudaMalloc((void **)&g->q32, (size_t)NQ32 * P * sizeof(float)) != cudaSuccess) ||
        cudaMalloc(&g->pairs, npairs * d) != cudaSuccess || cudaMalloc(&g->iflux, nflux * d) != cudaSuccess ||
        cudaMalloc((void **)&g->red, (size_t)NRED * nprob * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void **)&g->ds, (size_t)nprob * sizeof(DtSolve)) != cudaSuccess ||
        cudaMalloc((void **)&g->status, 2 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void **)&g->pin, std::max<size_t>(16, 3 * (size_t)nprob) * sizeof(double)) != cudaSuccess) {
        release(g);
        return ESMM_ERR_CUDA;
    }
    if (nprob > 1) {
        if (cudaMalloc((void **)&g->dpd, nprob * sizeof(ProbDesc)) != cudaSuccess ||
            cudaMemcpyAsync(g->dpd, g->hpd.data(), nprob * sizeof(ProbDesc), cudaMemcpyHostToDevice, g->st) !=
                cudaSuccess) {
            release(g);
            return ESMM_ERR_CUDA;
        }
    }
    // cold pressure guesses (NaN: the bracket midpoint), zero time and status
    bool ok = true;
    for (int k = 0; k < 3; ++k) ok = ok && cudaMemsetAsync(g->pg[k], 0xff, N * d, g->st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->status, 0, 2 * sizeof(int), g->st) == cudaSuccess &&
         cudaMemsetAsync(g->t_dev, 0, nprob * d, g->st) == cudaSuccess &&
         cudaStreamSynchronize(g->st) == cudaSuccess;
    if (!ok) { release(g); return ESMM_ERR_CUDA; }
    if (mesh_sweeps_init(g)) {
        release(g);
        return ESMM_ERR_CUDA;
    }
    *out = g;
    return ESMM_OK;
}

int check_geometry(int n0, int n1, const double *lo, const double *hi, const int *bc)
{
    const int n[2] = {n0, n1};
    for (int k = 0; k < 2; ++k) {
        if (n[k] < 4 || n[k] > (1 << 15)) return ESMM_ERR_ARG;
        if (bc[k] != ESMM_PERIODIC && bc[k] != ESMM_OUTFLOW && bc[k] != ESMM_INFLOW) return ESMM_ERR_ARG;
        if (!(hi[k] > lo[k])) return ESMM_ERR_ARG;
    }
    return ESMM_OK;
}

// state of problem b from primitive variables and a mesh (x NULL: uniform)
int state_set_one(esmm_grid *g, int b, const double *prim, const double *x, int mem)
{
    const ProbDesc &D = g->hpd[b];
    const Geom &G = D.g;
    size_t N = (size_t)G.N;
    double *xb = g->x + 2 * D.on;
    if (x) {
        int rc = copy_in(g, xb, x, 2 * N, mem);
        if (rc) return rc;
    } else {
        std::vector<double> hx(2 * N);
        int nx_ = G.bc0 == ESMM_PERIODIC ? G.nx : G.nx - 1;
        int ny_ = G.bc1 == ESMM_PERIODIC ? G.ny : G.ny - 1;
        const double *lo = &g->lo[2 * b], *hi = &g->hi[2 * b];
        for (int j = 0; j < G.ny; ++j)
            for (int i = 0; i < G.nx; ++i) {
                hx[(size_t)j * G.nx + i] = lo[0] + (hi[0] - lo[0]) * i / nx_;
                hx[N + (size_t)j * G.nx + i] = lo[1] + (hi[1] - lo[1]) * j / ny_;
            }
        CK(cudaMemcpyAsync(xb, hx.data(), 2 * N * sizeof(double), cudaMemcpyHostToDevice, g->st));
        CK(cudaStreamSynchronize(g->st));
    }
    // stage the primitives in the problem's slice of out_dc
    int rc = copy_in(g, g->out_dc + (size_t)g->nv * D.on, prim, (size_t)g->nv * N, mem);
    if (rc) return rc;
    CK(cudaMemsetAsync(g->status, 0, 2 * sizeof(int), g->st));
    LaunchDom L = dom_one(g, b, D_NODE);
    {
        Prof pr_(g, ESMM_KIND_NODE);
        if (g->phys == ESMM_RMHD)
            launch_init_mhd(L, g->p, g->gamma, g->out_dc, g->x, g->cons, g->J, g->status, g->st);
        else if (g->p == 1)
            k_init_state<1><<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->gamma, g->out_dc, g->x, g->cons, g->J, g->status);
        else if (g->p == 2)
            k_init_state<2><<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->gamma, g->out_dc, g->x, g->cons, g->J, g->status);
        else
            k_init_state<3><<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->gamma, g->out_dc, g->x, g->cons, g->J, g->status);
    }
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(g->xdot + 2 * D.on, 0, 2 * N * sizeof(double), g->st));
    for (int k = 0; k < 3; ++k) CK(cudaMemsetAsync(g->pg[k] + D.on, 0xff, N * sizeof(double), g->st));
    CK(cudaMemsetAsync(g->t_dev + b, 0, sizeof(double), g->st));
    int h[2];
    CK(cudaMemcpyAsync(h, g->status, sizeof h, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    g->xdot_zero = 1;
    if (h[1] > 0) {
        CK(cudaMemsetAsync(g->status, 0, 2 * sizeof(int), g->st));
        return fail(g, ESMM_ERR_ARG, "non-admissible initial state or tangled mesh");
    }
    return ESMM_OK;
}

int state_get_one(esmm_grid *g, int b, int what, double *out, int mem)
{
    const ProbDesc &D = g->hpd[b];
    size_t N = (size_t)D.g.N;
    int rc = ESMM_OK;
    switch (what) {
    case ESMM_GET_PRIM: {
        LaunchDom L = dom_one(g, b, D_NODE);
        {
            Prof pr_(g, ESMM_KIND_NODE);
            if (g->phys == ESMM_RMHD)
                launch_prim_out_mhd(L, g->gamma, g->cons, g->J, g->out_dc, g->status, g->st);
            else
                k_prim_out<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->gamma, g->cons, g->J, g->out_dc, g->status);
        }
        CK(cudaGetLastError());
        rc = copy_out(g, out, g->out_dc + (size_t)g->nv * D.on, (size_t)g->nv * N, mem);
        break;
    }
    case ESMM_GET_CONS: rc = copy_out(g, out, g->cons + (size_t)g->nv * D.on, (size_t)g->nv * N, mem); break;
    case ESMM_GET_J: rc = copy_out(g, out, g->J + D.on, N, mem); break;
    case ESMM_GET_X: rc = copy_out(g, out, g->x + 2 * D.on, 2 * N, mem); break;
    case ESMM_GET_XDOT: rc = copy_out(g, out, g->xdot + 2 * D.on, 2 * N, mem); break;
    default: return fail(g, ESMM_ERR_ARG, "unknown field");
    }
    if (rc) return rc;
    CK(cudaStreamSynchronize(g->st));
    if (what == ESMM_GET_PRIM) return check_c2p(g);
    return ESMM_OK;
}

// totals of every problem into tot_dev [nprob][3]
int totals_async(esmm_grid *g)
{
    int rc;
    if ((rc = ensure_doms(g))) return rc;
    node(g, g->cons, g->J, g->x, nullptr, nullptr, nullptr, true);
    LaunchDom L = dom(g, D_NODE);
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_totals<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->gamma, g->q, g->cons, g->J, g->partials);
    }
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_totals_final<<<nblk(3 * (long long)g->nprob, 128), 128, 0, g->st>>>(g->nprob, (int)L.nblk, L.pa.tiles,
                                                                               g->partials, g->tot_dev);
    }
    CK(cudaGetLastError());
    return ESMM_OK;
}

// kernels of one step, per profiling kind (for the launch count of graph replays)
void step_launches(const esmm_grid *g, double dt, long long per[ESMM_NKINDS])
{
    for (int k = 0; k < ESMM_NKINDS; ++k) per[k] = 0;
    per[ESMM_KIND_NODE] = 4;                       // 3 node passes + temporal metrics
    per[ESMM_KIND_PAIRS] = g->phys == ESMM_RMHD ? 0 : 6;
    per[ESMM_KIND_IFACE] = 6;
    per[ESMM_KIND_UPDATE] = 3;
    const int mu = g->prm.mu;
    const int sweeps = g->prm.precision == ESMM_MIXED ? (mu + MT_SB32 - 1) / MT_SB32 : (mu > 0) + mu;   // (+ residual)
    per[ESMM_KIND_MESH] = g->prm.move_mesh ? (4 + g->prm.n_filter + (mu > 0) + sweeps) : 0;
    // reset, (CFL), dt, time, and the Newton evaluations of a CFL step with mesh motion
    per[ESMM_KIND_OTHER] = 3 + (dt > 0.0 ? 0 : 1) + (g->prm.move_mesh && !(dt > 0.0) ? DT_NEWTON : 0);
}

// Advance every problem nsteps steps.  On a capturable stream one step is
// captured into a CUDA graph and replayed (the pressure warm-start buffers
// rotate back to the same assignment every step, so one graph serves any
// number of steps).
int advance(esmm_grid *g, int nsteps, double dt)
{
    int rc;
    if ((rc = ensure_doms(g))) return rc;
    bool capturable = g->st != nullptr && g->st != cudaStreamLegacy && g->st != cudaStreamPerThread &&
                      !(g->prm.move_mesh == 0 && !g->xdot_zero);
    const bool have = g->graph && g->graph_dt == dt && g->graph_epoch == g->epoch && g->graph_prof == g->prof_mask;
    // one step replays an existing graph; a new one is captured for two or more
    if (!capturable || (nsteps < 2 && !have)) {
        for (int s = 0; s < nsteps; ++s)
            if ((rc = rk_step_async(g, dt))) return rc;
        return ESMM_OK;
    }
    if (!have) {
        drop_graph(g);
        long long before[ESMM_NKINDS];
        memcpy(before, g->launches, sizeof before);
        cudaGraph_t gr = nullptr;
        CK(cudaStreamBeginCapture(g->st, cudaStreamCaptureModeThreadLocal));
        g->capturing = 1;
        rc = rk_step_async(g, dt);
        g->capturing = 0;
        cudaError_t e = cudaStreamEndCapture(g->st, &gr);
        memcpy(g->launches, before, sizeof before);
        if (rc) {
            if (gr) cudaGraphDestroy(gr);
            return rc;
        }
        if (e != cudaSuccess) return fail(g, ESMM_ERR_CUDA, "graph capture", e);
        e = cudaGraphInstantiate(&g->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) {
            g->graph = nullptr;
            return fail(g, ESMM_ERR_CUDA, "graph instantiate", e);
        }
        g->graph_dt = dt;
        g->graph_epoch = g->epoch;
        g->graph_prof = g->prof_mask;
    }
    long long per[ESMM_NKINDS];
    step_launches(g, dt, per);
    bool timed = false;
    for (int k = 0; k < ESMM_NKINDS; ++k) timed = timed || !g->gev[k].empty();
    for (int s = 0; s < nsteps; ++s) {
        // a profiled graph re-records its events: read the last replay's first
        if ((rc = collect_graph_prof(g))) return rc;
        CK(cudaGraphLaunch(g->graph, g->st));
        g->gev_pending = timed;
        for (int k = 0; k < ESMM_NKINDS; ++k) g->launches[k] += per[k];
    }
    return ESMM_OK;
}

// Autotuner: for each kernel kind, time the candidate block sizes (and, for
// batches, the tile orders natural / largest-first) on the current state and
// keep the fastest.
int tune(esmm_grid *g)
{
    int rc;
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    if ((rc = ensure_doms(g))) return rc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int saved_mask = g->prof_mask;
    long long saved_launches[ESMM_NKINDS];
    memcpy(saved_launches, g->launches, sizeof saved_launches);
    g->prof_mask = 0;
    auto time_it = [&](auto &&fn) -> float {
        fn();   // warm-up
        cudaEventRecord(e0, g->st);
        fn();
        fn();
        cudaEventRecord(e1, g->st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    auto run_node = [&]() { node(g, g->cons, g->J, g->x, g->xdot, nullptr, nullptr); };
    run_node();
    struct Cand { int kind; int kind2; std::vector<int> bs; };
    std::vector<Cand> cands = {{D_PAD, D_PAD, {128, 256, 512}},
                               {D_NODE, D_NODE2, {128, 256, 512}}};
    if (g->phys == ESMM_RMHD) cands.push_back({D_IFACE0, D_IFACE1, {64, 128}});
    Phys ph = phys(g);
    bool f32 = g->prm.precision == ESMM_MIXED;
    if (g->phys == ESMM_RHD) {
        // the tiled pair and interface launches, each direction on its own:
        // block size x tile shape (flat runs, or tx sites along x_1 by bs / tx
        // along x_2) x one block per tile or a persistent grid (x the tile
        // order of a batch)
        for (int dir = 0; dir < 2; ++dir) {   // pair fluxes in place for the interface timings
            LaunchDom L = dom(g, dir ? D_TPAIR1 : D_TPAIR0);
            if (f32) launch_pairs_f32(L, ph, g->q, g->q32, g->pairs, dir, g->st);
            else launch_pairs_f64(L, ph, g->q, nullptr, g->pairs, dir, g->st);
        }
        float split_ms[2] = {0.0f, 0.0f};
        for (int kind = D_TPAIR0; kind <= D_TIFACE1; ++kind) {
            const int dir = (kind == D_TPAIR1 || kind == D_TIFACE1) ? 1 : 0;
            const bool pairs = kind <= D_TPAIR1;
            std::vector<int> orders = g->nprob > 1 ? std::vector<int>{0, 1} : std::vector<int>{0};
            float best = 1e30f;
            int bb = g->bs[kind], bt = g->tx[kind], bp = g->persist[kind], bo = g->order_lpt[kind];
            for (int bs : {64, 128})
                for (int tx : {0, 8, 16, 32, 64, 128}) {
                    if (tx > bs) continue;
                    for (int per : {0, 1})
                        for (int ord : orders) {
                            g->bs[kind] = bs;
                            g->tx[kind] = tx;
                            g->persist[kind] = per;
                            g->order_lpt[kind] = ord;
                            if ((rc = build_dom(g, kind))) return rc;
                            const float ms = time_it([&]() {
                                LaunchDom L = dom(g, kind);
                                if (pairs) {
                                    if (f32) launch_pairs_f32(L, ph, g->q, g->q32, g->pairs, dir, g->st);
                                    else launch_pairs_f64(L, ph, g->q, nullptr, g->pairs, dir, g->st);
                                } else {
                                    if (f32) launch_iface_f32(L, ph, g->q, g->q32, g->pairs, g->iflux, dir, g->st);
                                    else launch_iface_f64(L, ph, g->q, nullptr, g->pairs, g->iflux, dir, g->st);
                                }
                            });
                            if (ms < best) {
                                best = ms;
                                bb = bs;
                                bt = tx;
                                bp = per;
                                bo = ord;
                            }
                        }
                }
            g->bs[kind] = bb;
            g->tx[kind] = bt;
            g->persist[kind] = bp;
            g->order_lpt[kind] = bo;
            if ((rc = build_dom(g, kind))) return rc;
            split_ms[dir] += best;
        }
        // the fused sweep kernel against the best pair + interface launches,
        // per direction (unless the parameters fix the variant)
        for (int dir = 0; dir < 2 && g->prm.sweep != ESMM_SWEEP_SPLIT; ++dir) {
            const int kind = dir ? D_TIFACE1 : D_TIFACE0;
            std::vector<int> orders = g->nprob > 1 ? std::vector<int>{0, 1} : std::vector<int>{0};
            const int sb = g->bs[kind], st_ = g->tx[kind], sp = g->persist[kind], so = g->order_lpt[kind];
            float best = 1e30f;
            int bb = 128, bp = 0, bo = 0;
            for (int bs : {64, 128, 256})
                for (int per : {0, 1})
                    for (int ord : orders) {
                        g->bs[kind] = bs;
                        g->tx[kind] = -1;
                        g->persist[kind] = per;
                        g->order_lpt[kind] = ord;
                        if ((rc = build_dom(g, kind))) return rc;
                        const float ms = time_it([&]() {
                            LaunchDom L = dom(g, kind);
                            if (f32) launch_sweep_f32(L, ph, g->q, g->q32, g->iflux, dir, g->st);
                            else launch_sweep_f64(L, ph, g->q, nullptr, g->iflux, dir, g->st);
                        });
                        if (ms < best) {
                            best = ms;
                            bb = bs;
                            bp = per;
                            bo = ord;
                        }
                    }
            const bool fused = g->prm.sweep == ESMM_SWEEP_FUSED || best < split_ms[dir];
            g->bs[kind] = fused ? bb : sb;
            g->tx[kind] = fused ? -1 : st_;
            g->persist[kind] = fused ? bp : sp;
            g->order_lpt[kind] = fused ? bo : so;
            if ((rc = build_dom(g, kind))) return rc;
        }
    }
    for (auto &c : cands) {
        std::vector<int> orders = g->nprob > 1 ? std::vector<int>{0, 1} : std::vector<int>{0};
        float best = 1e30f;
        int best_bs = g->bs[c.kind], best_ord = g->order_lpt[c.kind];
        for (int bs : c.bs)
            for (int ord : orders) {
                for (int k : {c.kind, c.kind2}) {
                    g->bs[k] = bs;
                    g->order_lpt[k] = ord;
                    if ((rc = build_dom(g, k))) return rc;
                }
                float ms;
                if (c.kind == D_PAD) {
                    ms = time_it(run_node);
                } else if (c.kind == D_NODE) {
                    ms = time_it([&]() {
                        update(g, g->out_dc, g->out_dJ, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                               nullptr, 0.0, 0.0, nullptr, nullptr, nullptr);
                    });
                } else if (g->phys == ESMM_RMHD) {
                            ms = c.kind == D_PAIR0 ? 0.0f : time_it([&]() {
                                for (int dir = 0; dir < 2; ++dir)
                                    if (f32)
                                        launch_iface_mhd_f32(dom(g, dir ? c.kind2 : c.kind), ph, g->q, g->iflux,
                                                             dir, g->st);
                                    else
                                        launch_iface_mhd(dom(g, dir ? c.kind2 : c.kind), ph, g->q, g->iflux, dir,
                                                         g->st);
                            });
                } else {
                    ms = time_it([&]() {
                        for (int dir = 0; dir < 2; ++dir) {
                            LaunchDom L = dom(g, dir ? c.kind2 : c.kind);
                            if (c.kind == D_PAIR0) {
                                if (f32) launch_pairs_f32(L, ph, g->q, g->q32, g->pairs, dir, g->st);
                                else launch_pairs_f64(L, ph, g->q, nullptr, g->pairs, dir, g->st);
                            } else {
                                if (f32) launch_iface_f32(L, ph, g->q, g->q32, g->pairs, g->iflux, dir, g->st);
                                else launch_iface_f64(L, ph, g->q, nullptr, g->pairs, g->iflux, dir, g->st);
                            }
                        }
                    });
                }
                if (ms < best) { best = ms; best_bs = bs; best_ord = ord; }
            }
        for (int k : {c.kind, c.kind2}) {
            g->bs[k] = best_bs;
            g->order_lpt[k] = best_ord;
            if ((rc = build_dom(g, k))) return rc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g->prof_mask = saved_mask;
    memcpy(g->launches, saved_launches, sizeof saved_launches);
    g->tuned = 1;
    g->epoch++;
    CK(cudaGetLastError());
    return ESMM_OK;
}

// ---- adjoint -------------------------------------------------------------------
int adj_alloc(esmm_grid *g)
{
    size_t P = (size_t)g->Ptot, N = (size_t)g->Ntot, d = sizeof(double);
    if (!g->adjG) CK(cudaMalloc((void **)&g->adjG, ADJ_G_PER_NODE * P * d));
    if (!g->adjGp) CK(cudaMalloc((void **)&g->adjGp, ADJ_GP_PER_NODE * P * d));
    double **bufs[] = {&g->lam_a, &g->lam_b, &g->lam_c, &g->lam_v};
    for (double **b : bufs)
        if (!*b) CK(cudaMalloc((void **)b, (size_t)g->nv * N * d));
    return ESMM_OK;
}

// lam = (d rhs/d cons)^T mu at (cons, J, x, xdot), all device arrays
int rhs_vjp_core(esmm_grid *g, const double *cons, const double *J, const double *x, const double *xdot,
                 const double *mu, double *lam)
{
    size_t P = (size_t)g->Ptot, N = (size_t)g->Ntot, d = sizeof(double);
    node(g, cons, J, x, xdot, nullptr, nullptr);
    if (g->phys == ESMM_RMHD) {
        // forward interface fluxes first: the Powell term needs div B~
        fluxes(g);
        CK(cudaMemsetAsync(g->adjG, 0, ADJ_LAMQ_PER_NODE * P * d, g->st));
        CK(cudaMemsetAsync(lam, 0, 8 * N * d, g->st));
        Phys ph = phys(g);
        for (int dir = 0; dir < 2; ++dir) {
            {
                Prof pr_(g, ESMM_KIND_PAIRS);
                launch_pairs_vjp_mhd(dom(g, dir ? D_PAIR1 : D_PAIR0), ph, g->q, mu, g->adjG, dir, g->st);
            }
            if (g->w > 0) {
                Prof pr_(g, ESMM_KIND_IFACE);
                launch_iface_vjp_mhd(dom(g, dir ? D_IFACE1 : D_IFACE0), ph, g->q, mu, g->adjG, dir, g->st);
            }
        }
        {
            Prof pr_(g, ESMM_KIND_NODE);
            launch_node_vjp_mhd(dom(g, D_PAD), g->gamma, g->q, g->adjG, (const double *)g->iflux, mu, J, lam,
                                g->st);
        }
        CK(cudaGetLastError());
        return ESMM_OK;
    }
    CK(cudaMemsetAsync(g->adjG, 0, ADJ_G_PER_NODE * P * d, g->st));
    CK(cudaMemsetAsync(g->adjGp, 0, ADJ_GP_PER_NODE * P * d, g->st));
    CK(cudaMemsetAsync(lam, 0, 4 * N * d, g->st));
    Phys ph = phys(g);
    for (int dir = 0; dir < 2; ++dir) {
        {
            Prof pr_(g, ESMM_KIND_PAIRS);
            launch_pairs_vjp(dom(g, dir ? D_PAIR1 : D_PAIR0), ph, g->q, mu, g->adjGp, dir, g->st);
        }
        if (g->w > 0) {
            Prof pr_(g, ESMM_KIND_IFACE);
            launch_iface_vjp(dom(g, dir ? D_IFACE1 : D_IFACE0), ph, g->q, mu, g->adjG, dir, g->st);
        }
    }
    {
        Prof pr_(g, ESMM_KIND_NODE);
        launch_node_vjp(dom(g, D_PAD), g->gamma, g->p, g->w, g->q, g->adjG, g->adjGp, J, lam, g->st);
    }
    CK(cudaGetLastError());
    return ESMM_OK;
}

int set_dt(esmm_grid *g, double dt)
{
    g->pin[0] = dt;
    CK(cudaMemcpyAsync(g->dt_dev, g->pin, sizeof(double), cudaMemcpyHostToDevice, g->st));
    CK(cudaStreamSynchronize(g->st));
    return ESMM_OK;
}

// One step with a given mesh velocity ([2][N], host or device) and dt: the
// map the adjoint differentiates, and the prescribed mesh motion.
int step_given(esmm_grid *g, const double *xd, double dt, int mem)
{
    int rc;
    if ((rc = ensure_doms(g)) || (rc = set_dt(g, dt))) return rc;
    if ((rc = copy_in(g, g->xdot, xd, 2 * (size_t)g->Ntot, mem))) return rc;
    g->xdot_zero = 0;
    node(g, g->cons, g->J, g->x, g->xdot, g->pg[0], g->pg[1]);
    return stages(g);
}

}  // namespace

// ---------------------------------------------------------------------------
// Slabs of a decomposed grid (esmm_slab_create).  A slab is a one-problem
// grid of its held rows; its reductions collect its own rows only, and the
// host combines them over the slabs through the caller's comm between the
// kernels that need the combined values.
namespace {

double host_bits(unsigned long long b)
{
    double v;
    memcpy(&v, &b, sizeof v);
    return v;
}
unsigned long long host_to_bits(double v)
{
    unsigned long long b;
    memcpy(&b, &v, sizeof b);
    return b;
}

int slab_allreduce(esmm_grid *g, double *buf, int n, int op)
{
    if (n > 0 && g->comm.allreduce(g->comm.ctx, buf, n, op) != 0)
        return fail(g, ESMM_ERR_CUDA, "slab allreduce failed");
    return ESMM_OK;
}

// combine the reduction slots in mx by max and those in mn by min over the
// slabs (in place on the device)
int slab_slots(esmm_grid *g, std::initializer_list<int> mx, std::initializer_list<int> mn)
{
    unsigned long long h[NRED];
    CK(cudaMemcpyAsync(h, g->red, sizeof h, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    double b[NRED];
    int k = 0, rc;
    for (int i : mx) b[k++] = host_bits(h[i]);
    if ((rc = slab_allreduce(g, b, k, ESMM_OP_MAX))) return rc;
    k = 0;
    for (int i : mx) h[i] = host_to_bits(b[k++]);
    k = 0;
    for (int i : mn) b[k++] = host_bits(h[i]);
    if ((rc = slab_allreduce(g, b, k, ESMM_OP_MIN))) return rc;
    k = 0;
    for (int i : mn) h[i] = host_to_bits(b[k++]);
    CK(cudaMemcpyAsync(g->red, h, sizeof h, cudaMemcpyHostToDevice, g->st));
    CK(cudaStreamSynchronize(g->st));
    return ESMM_OK;
}

// one array [ncomp][N] of the slab to exchange; shift: the component that
// moves by the period where a halo crosses the periodic seam (-1: none)
struct XArr {
    double *p;
    int ncomp, shift;
};

// Halo exchange: the slab's lowest and highest ESMM_SLAB_HALO own rows of
// every array go to the neighbours below and above, whose own rows fill the
// slab's halo rows.
int slab_exchange(esmm_grid *g, std::initializer_list<XArr> arrs)
{
    const Geom &G = g->hpd[0].g;
    const long long H = ESMM_SLAB_HALO, row = G.nx, N = G.N, blk = H * row;
    size_t count = 0;
    for (const XArr &a : arrs) count += (size_t)a.ncomp * blk;
    if (count > g->xbuf_n) {
        if (g->xbuf) cudaFreeHost(g->xbuf);
        g->xbuf = nullptr;
        g->xbuf_n = 0;
        CK(cudaMallocHost((void **)&g->xbuf, 4 * count * sizeof(double)));
        g->xbuf_n = count;
    }
    double *slo = g->xbuf, *shi = slo + count, *rlo = shi + count, *rhi = rlo + count;
    const bool lo = g->ext0 < g->own0, hi = g->ext1 > g->own1;
    const long long o0 = g->own0 - g->ext0, o1 = g->own1 - g->ext0;
    long long off = 0;
    for (const XArr &a : arrs)
        for (int c = 0; c < a.ncomp; ++c, off += blk) {
            if (lo) CK(cudaMemcpyAsync(slo + off, a.p + c * N + o0 * row, blk * sizeof(double),
                                       cudaMemcpyDeviceToHost, g->st));
            if (hi) CK(cudaMemcpyAsync(shi + off, a.p + c * N + (o1 - H) * row, blk * sizeof(double),
                                       cudaMemcpyDeviceToHost, g->st));
        }
    CK(cudaStreamSynchronize(g->st));
    if (g->comm.exchange(g->comm.ctx, lo ? slo : nullptr, hi ? shi : nullptr, lo ? rlo : nullptr,
                         hi ? rhi : nullptr, (long long)count) != 0)
        return fail(g, ESMM_ERR_CUDA, "slab halo exchange failed");
    off = 0;
    for (const XArr &a : arrs)
        for (int c = 0; c < a.ncomp; ++c, off += blk) {
            if (c == a.shift && g->periodic1) {   // halos across the periodic seam
                if (lo && g->slab == 0)
                    for (long long q = 0; q < blk; ++q) rlo[off + q] -= g->per1;
                if (hi && g->slab == g->nslab - 1)
                    for (long long q = 0; q < blk; ++q) rhi[off + q] += g->per1;
            }
            if (lo) CK(cudaMemcpyAsync(a.p + c * N + (o0 - H) * row, rlo + off, blk * sizeof(double),
                                       cudaMemcpyHostToDevice, g->st));
            if (hi) CK(cudaMemcpyAsync(a.p + c * N + o1 * row, rhi + off, blk * sizeof(double),
                                       cudaMemcpyHostToDevice, g->st));
        }
    CK(cudaStreamSynchronize(g->st));
    return ESMM_OK;
}

int slab_exchange_state(esmm_grid *g, double *cons, double *J, double *x)
{
    return slab_exchange(g, {{cons, g->nv, -1}, {J, 1, -1}, {x, 2, 1}});
}

// The step of eq. cfl on a slab: the Newton evaluations of the solve, each
// combined over the slabs (max of each direction's value, then min of the
// slope among the slabs that attain it: the undecomposed rule), with the
// update of esmm_reduce.cuh applied on the host.
int slab_newton(esmm_grid *g)
{
    DtSolve S;
    CK(cudaMemcpyAsync(&S, g->ds, sizeof S, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    LaunchDom L = dom(g, D_NEWTON);
    double *vs_dev = g->vs_dev;
    if (S.done) return ESMM_OK;   // ended in the set-up (no mesh motion): dt_dev holds the step
    double dt = 0.0;
    int rc = ESMM_OK;
    while (!S.done) {
        {
            Prof pr_(g, ESMM_KIND_OTHER);
            k_dt_newton<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->prm.cfl, g->cflb, g->red, g->ds, g->npart, g->dt_dev,
                                                    vs_dev);
        }
        double h[4];
        if (cudaMemcpyAsync(h, vs_dev, sizeof h, cudaMemcpyDeviceToHost, g->st) != cudaSuccess ||
            cudaStreamSynchronize(g->st) != cudaSuccess) {
            rc = fail(g, ESMM_ERR_CUDA, "slab Newton read-back");
            break;
        }
        double V[2] = {h[0], h[2]}, Sl[2];
        if ((rc = slab_allreduce(g, V, 2, ESMM_OP_MAX))) break;
        for (int k = 0; k < 2; ++k) Sl[k] = h[2 * k] == V[k] ? h[2 * k + 1] : HUGE_VAL;
        if ((rc = slab_allreduce(g, Sl, 2, ESMM_OP_MIN))) break;
        double gsum = 0.0, slope = 0.0;
        for (int k = 0; k < 2; ++k) {
            gsum += V[k];
            slope += Sl[k];
        }
        dt_newton_update(&S, gsum, slope, g->prm.cfl, &dt);
        if (cudaMemcpyAsync(g->ds, &S, sizeof S, cudaMemcpyHostToDevice, g->st) != cudaSuccess ||
            cudaStreamSynchronize(g->st) != cudaSuccess) {
            rc = fail(g, ESMM_ERR_CUDA, "slab Newton update");
            break;
        }
    }
    if (rc) return rc;
    g->pin[0] = dt;
    CK(cudaMemcpyAsync(g->dt_dev, g->pin, sizeof(double), cudaMemcpyHostToDevice, g->st));
    CK(cudaStreamSynchronize(g->st));
    return ESMM_OK;
}

// State of a slab from the GLOBAL arrays (host): its held rows, with the
// periodic wrap (rows beyond an end shifted by the period in x_2), then a
// halo exchange so that the halo rows' J and cons are the neighbours' (the
// slab's own set-up differences them at its cuts).
int slab_state_set(esmm_grid *g, const double *prim, const double *x, int mem)
{
    if (mem != ESMM_MEM_HOST) return fail(g, ESMM_ERR_ARG, "a slab's state is set from host arrays");
    const Geom &G = g->hpd[0].g;
    const size_t nx = (size_t)G.nx, nyl = (size_t)G.ny, Nl = nx * nyl, Ng = nx * (size_t)g->rows_g;
    std::vector<double> hp((size_t)g->nv * Nl), hx(x ? 2 * Nl : 0);
    for (size_t r = 0; r < nyl; ++r) {
        const long long gr = g->ext0 + (long long)r;
        const long long src = ((gr % g->rows_g) + g->rows_g) % g->rows_g;
        const double shift = (double)((gr - src) / g->rows_g) * g->per1;
        for (int c = 0; c < g->nv; ++c)
            memcpy(&hp[c * Nl + r * nx], prim + c * Ng + src * nx, nx * sizeof(double));
        if (x) {
            memcpy(&hx[r * nx], x + src * nx, nx * sizeof(double));
            for (size_t i = 0; i < nx; ++i) hx[Nl + r * nx + i] = x[Ng + src * nx + i] + shift;
        }
    }
    int rc = state_set_one(g, 0, hp.data(), x ? hx.data() : nullptr, ESMM_MEM_HOST);
    int rx = slab_exchange_state(g, g->cons, g->J, g->x);   // collective: every slab exchanges
    return rc ? rc : rx;
}

// the slab's own rows of one field
int slab_state_get(esmm_grid *g, int what, double *out, int mem)
{
    const Geom &G = g->hpd[0].g;
    const size_t nx = (size_t)G.nx, Nl = (size_t)G.N, rows = (size_t)(g->own1 - g->own0);
    const size_t o0 = (size_t)(g->own0 - g->ext0) * nx;
    int nc = (what == ESMM_GET_PRIM || what == ESMM_GET_CONS) ? g->nv : (what == ESMM_GET_J ? 1 : 2);
    const double *src = nullptr;
    int rc = ESMM_OK;
    switch (what) {
    case ESMM_GET_PRIM: {
        LaunchDom L = dom_one(g, 0, D_NODE);
        {
            Prof pr_(g, ESMM_KIND_NODE);
            if (g->phys == ESMM_RMHD)
                launch_prim_out_mhd(L, g->gamma, g->cons, g->J, g->out_dc, g->status, g->st);
            else
                k_prim_out<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->gamma, g->cons, g->J, g->out_dc, g->status);
        }
        src = g->out_dc;
        break;
    }
    case ESMM_GET_CONS: src = g->cons; break;
    case ESMM_GET_J: src = g->J; break;
    case ESMM_GET_X: src = g->x; break;
    case ESMM_GET_XDOT: src = g->xdot; break;
    default: return fail(g, ESMM_ERR_ARG, "unknown field");
    }
    for (int c = 0; c < nc && !rc; ++c) rc = copy_out(g, out + c * rows * nx, src + c * Nl + o0, rows * nx, mem);
    if (rc) return rc;
    CK(cudaStreamSynchronize(g->st));
    return what == ESMM_GET_PRIM ? check_c2p(g) : ESMM_OK;
}

// One step of a slab (synchronous: the reductions and exchanges go through
// the host).  The kernels are those of rk_step_async; only the points where
// a combined value is needed differ.
int slab_step(esmm_grid *g, double dt)
{
    int rc;
    if ((rc = ensure_doms(g))) return rc;
    const bool moving = g->prm.move_mesh, solve = moving && !(dt > 0.0);
    node(g, g->cons, g->J, g->x, nullptr, g->pg[0], g->pg[1]);
    red_init(g);
    step_radius(g, dt, moving);
    LaunchDom L = dom(g, D_NODE), L2 = dom(g, D_NODE2);
    if (moving) {
        Prof pr_(g, ESMM_KIND_MESH);
        k_mesh_grad<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->prm.monitor == ESMM_MONITOR_LNRHO, g->prm.alpha_lap > 0.0,
                                                g->q, g->grad, g->om2, g->red);
    }
    if ((rc = slab_slots(g, {0, 2, 3, 6}, {}))) return rc;
    if (!moving) {
        step_dt(g, dt, false);
        if (!g->xdot_zero) {
            CK(cudaMemsetAsync(g->xdot, 0, sizeof(double) * 2 * g->Ntot, g->st));
            g->xdot_zero = 1;
        }
    } else {
        g->xdot_zero = 0;
        {
            Prof pr_(g, ESMM_KIND_MESH);
            k_mesh_omega<<<L.nblk, L.bs, 0, g->st>>>(L.pa, g->prm.alpha, g->prm.alpha_lap, g->grad, g->om2, g->red,
                                                     g->om);
        }
        double *om = g->om, *om2 = g->om2;
        for (int f = 0; f < g->prm.n_filter; ++f) {
            Prof pr_(g, ESMM_KIND_MESH);
            k_mesh_filter<<<L.nblk, L.bs, 0, g->st>>>(L.pa, om, om2);
            std::swap(om, om2);
        }
        if (g->prm.mu > 0) {
            Prof pr_(g, ESMM_KIND_MESH);
            k_mesh_weights<<<L.nblk, L.bs, 0, g->st>>>(L.pa, om, g->cw);
        }
        // the sweeps and the limiter (mesh_finish without its dt and mesh velocity)
        const bool f32 = g->prm.precision == ESMM_MIXED;
        if (f32) rc = mesh_sweeps_tau<float, MT_SB32>(g, L);
        else rc = mesh_sweeps_tau<double, 1>(g, L);
        if (rc) return rc;
        if ((rc = slab_slots(g, {4, 5}, {1}))) return rc;
        {
            Prof pr_(g, ESMM_KIND_OTHER);
            k_dt<<<nprob_blocks(g), 128, 0, g->st>>>(g->nprob, g->prm.cfl, dt, g->red, g->ds, g->dt_dev);
        }
        if (solve && (rc = slab_newton(g))) return rc;
        {
            Prof pr_(g, ESMM_KIND_MESH);
            if (f32)
                k_mesh_xdot<float><<<L2.nblk, L2.bs, 0, g->st>>>(L2.pa, (const float *)g->mesh_disp, g->red,
                                                                 g->dt_dev, g->xdot);
            else
                k_mesh_xdot<double><<<L2.nblk, L2.bs, 0, g->st>>>(L2.pa, (const double *)g->mesh_disp, g->red,
                                                                  g->dt_dev, g->xdot);
        }
        if ((rc = slab_exchange(g, {{g->xdot, 2, -1}}))) return rc;
    }
    {
        Prof pr_(g, ESMM_KIND_NODE);
        LaunchDom Lp = dom(g, D_PAD);
        k_tmetric<<<Lp.nblk, Lp.bs, 0, g->st>>>(Lp.pa, g->xdot, g->q, q32_of(g));
    }
    fluxes(g);
    update(g, nullptr, nullptr, g->cons, g->J, g->x, g->cons, g->J, g->x, g->xdot, 0.0, 1.0, g->c1, g->J1, g->x1);
    if ((rc = slab_exchange_state(g, g->c1, g->J1, g->x1))) return rc;
    node(g, g->c1, g->J1, g->x1, g->xdot, g->pg[1], g->pg[2]);
    fluxes(g);
    update(g, nullptr, nullptr, g->cons, g->J, g->x, g->c1, g->J1, g->x1, g->xdot, 0.75, 0.25, g->c2, g->J2, g->x2);
    if ((rc = slab_exchange_state(g, g->c2, g->J2, g->x2))) return rc;
    node(g, g->c2, g->J2, g->x2, g->xdot, g->pg[2], g->pg[0]);
    fluxes(g);
    update(g, nullptr, nullptr, g->cons, g->J, g->x, g->c2, g->J2, g->x2, g->xdot, 1.0 / 3.0, 2.0 / 3.0, g->cons,
           g->J, g->x);
    if ((rc = slab_exchange_state(g, g->cons, g->J, g->x))) return rc;
    {
        Prof pr_(g, ESMM_KIND_OTHER);
        k_time<<<nprob_blocks(g), 128, 0, g->st>>>(g->nprob, g->dt_dev, g->t_dev);
    }
    CK(cudaGetLastError());
    return ESMM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Allocation-free right-hand side (esmm_rhs_static).
//
// Its scratch lives in one file-scope device array: per padded node the NQ
// node arrays, the pair fluxes [2][PMAX][4] and the interface fluxes [2][5]
// (48 doubles), then two status ints.  Every GPU that loads the library holds
// this array until the process exits.  Host code only ever passes the
// device address obtained from cudaGetSymbolAddress: in host code the
// array's name is a host-side stand-in, not a device address.
constexpr long long STATIC_PER_NODE = NQ + 2 * PMAX * 4 + 2 * 5;
constexpr long long STATIC_DOUBLES = STATIC_PER_NODE * ESMM_STATIC_MAX_PADDED_NODES + 32;
static __device__ __align__(256) double esmm_static_scratch[STATIC_DOUBLES];

namespace {
constexpr int STATIC_MAX_DEVICES = 64;
std::mutex static_mu;
double *static_ptr[STATIC_MAX_DEVICES];     // device address per device

// Device address of the scratch on the current device.  The first call on a
// device looks it up with that device current (with lazy module loading this
// is also when the driver reserves the array).  Later calls look it up again
// unless the stream is being captured, so an address made stale by a
// cudaDeviceReset (which reloads the module) is never used outside a capture;
// inside a capture the address cached by an earlier call is used, and a first
// call inside a capture is refused.
cudaError_t static_scratch(cudaStream_t st, double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= STATIC_MAX_DEVICES) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(static_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, esmm_static_scratch);
        if (e != cudaSuccess) return e;
        static_ptr[dev] = p;
    } else if (!static_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = static_ptr[dev];
    return cudaSuccess;
}
}  // namespace

// ===========================================================================
extern "C" {

int esmm_mhd_eigen(double gamma, int n, const double *w, const double *dw, double *lam, double *R, double *dlam,
                   double *dR)
{
    if (n < 1 || !w || !lam || !R || (dw && (!dlam || !dR))) return ESMM_ERR_ARG;
    return mhd_eigen_host(gamma, n, w, dw, lam, R, dlam, dR) ? ESMM_ERR_CUDA : ESMM_OK;
}

const char *esmm_version(void) { return "esmm 0.4 (2D RHD and RMHD, 3D RMHD, batched RHD, sm_103a)"; }

int esmm_grid_create(esmm_grid **out, int dim, const int n[3], const double lo[3], const double hi[3], int phys,
                     const int bc[3], void *stream)
{
    if (!out || !n || !lo || !hi || !bc) return ESMM_ERR_ARG;
    *out = nullptr;
    if (dim == 3) return phys == ESMM_RMHD ? create3(out, n, lo, hi, bc, stream) : ESMM_ERR_ARG;
    if (dim != 2 || (phys != ESMM_RHD && phys != ESMM_RMHD)) return ESMM_ERR_ARG;
    if (check_geometry(n[0], n[1], lo, hi, bc)) return ESMM_ERR_ARG;
    int n2[2] = {n[0], n[1]}, bc2[2] = {bc[0], bc[1]};
    double lo2[2] = {lo[0], lo[1]}, hi2[2] = {hi[0], hi[1]};
    return create(out, 1, n2, lo2, hi2, bc2, phys, stream, false);
}

int esmm_slab_create(esmm_grid **out, const int n[2], const double lo[2], const double hi[2], int phys,
                     const int bc[2], int nslab, int slab, const esmm_comm *comm, void *stream)
{
    if (!out || !n || !lo || !hi || !bc || !comm || !comm->allreduce || !comm->exchange) return ESMM_ERR_ARG;
    *out = nullptr;
    if ((phys != ESMM_RHD && phys != ESMM_RMHD) || check_geometry(n[0], n[1], lo, hi, bc)) return ESMM_ERR_ARG;
    if (bc[0] == ESMM_INFLOW || bc[1] == ESMM_INFLOW) return ESMM_ERR_ARG;
    const int H = ESMM_SLAB_HALO, ny = n[1];
    if (nslab < 2 || slab < 0 || slab >= nslab || ny / nslab < H) return ESMM_ERR_ARG;
    const int base = ny / nslab, rem = ny % nslab;
    const int own0 = slab * base + std::min(slab, rem), own1 = own0 + base + (slab < rem ? 1 : 0);
    const bool per = bc[1] == ESMM_PERIODIC;
    const int ext0 = (slab > 0 || per) ? own0 - H : own0, ext1 = (slab < nslab - 1 || per) ? own1 + H : own1;
    // the held rows as an outflow grid whose uniform mesh is the whole grid's
    const double dy = (hi[1] - lo[1]) / (per ? ny : ny - 1);
    int nl[2] = {n[0], ext1 - ext0}, bcl[2] = {bc[0], ESMM_OUTFLOW};
    double lol[2] = {lo[0], lo[1] + ext0 * dy}, hil[2] = {hi[0], lo[1] + (ext1 - 1) * dy};
    esmm_grid *g = nullptr;
    int rc = create(&g, 1, nl, lol, hil, bcl, phys, stream, false);
    if (rc) return rc;
    g->nslab = nslab;
    g->slab = slab;
    g->comm = *comm;
    g->rows_g = ny;
    g->own0 = own0;
    g->own1 = own1;
    g->ext0 = ext0;
    g->ext1 = ext1;
    g->periodic1 = per;
    g->per1 = hi[1] - lo[1];
    g->hpd[0].g.own0 = own0 - ext0;
    g->hpd[0].g.own1 = own1 - ext0;
    if (cudaMalloc((void **)&g->vs_dev, 4 * sizeof(double)) != cudaSuccess) {
        release(g);
        return ESMM_ERR_CUDA;
    }
    *out = g;
    return ESMM_OK;
}

int esmm_slab_rows(const esmm_grid *g, int *own0, int *own1, int *ext0, int *ext1)
{
    if (!g || g->nslab == 0) return ESMM_ERR_ARG;
    if (own0) *own0 = g->own0;
    if (own1) *own1 = g->own1;
    if (ext0) *ext0 = g->ext0;
    if (ext1) *ext1 = g->ext1;
    return ESMM_OK;
}

int esmm_grid_destroy(esmm_grid *g)
{
    if (!g) return ESMM_ERR_ARG;
    cudaStreamSynchronize(g->st);
    release(g);
    return ESMM_OK;
}

int esmm_set_stream(esmm_grid *g, void *stream)
{
    if (!g) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_set_stream(g->g3, stream);
    CK(cudaStreamSynchronize(g->st));
    g->st = stream ? (cudaStream_t)stream : (g->own_st ? g->own_st : nullptr);
    drop_graph(g);
    return ESMM_OK;
}

int esmm_set_eos(esmm_grid *g, double gamma)
{
    if (!g || !(gamma > 1.0 && gamma <= 2.0)) return fail(g, ESMM_ERR_ARG, "Gamma must be in (1, 2]");
    if (g->dim == 3) return esmm3_set_eos(g->g3, gamma);
    g->gamma = gamma;
    g->epoch++;
    return ESMM_OK;
}

int esmm_set_order(esmm_grid *g, int p, int w)
{
    if (!g || p < 1 || p > PMAX || !(w == 0 || w == 3 || w == 5))
        return fail(g, ESMM_ERR_ARG, "p must be 1..3 and w one of 0, 3, 5");
    if (g->dim == 3) return esmm3_set_order(g->g3, p, w);
    if (p != g->p) g->doms_valid = 0;
    g->p = p;
    g->w = w;
    g->epoch++;
    return ESMM_OK;
}

int esmm_set_params(esmm_grid *g, const esmm_params *prm)
{
    if (!g || !prm) return ESMM_ERR_ARG;
    if (!(prm->cfl > 0.0) || !(prm->weno_eps > 0.0) || !(prm->alpha >= 0.0) || !(prm->alpha_lap >= 0.0) ||
        prm->n_filter < 0 ||
        prm->mu < 0 || (prm->precision != ESMM_FP64 && prm->precision != ESMM_MIXED) ||
        (prm->monitor != ESMM_MONITOR_RHO && prm->monitor != ESMM_MONITOR_LNRHO))
        return fail(g, ESMM_ERR_ARG, "invalid parameter");
    if (prm->sweep != ESMM_SWEEP_AUTO && prm->sweep != ESMM_SWEEP_FUSED && prm->sweep != ESMM_SWEEP_SPLIT)
        return fail(g, ESMM_ERR_ARG, "invalid parameter");
    if (g->dim == 3) return esmm3_set_params(g->g3, prm);
    if (prm->sweep != g->prm.sweep) set_sweep(g, prm->sweep);
    g->prm = *prm;
    g->epoch++;
    return ESMM_OK;
}

int esmm_get_params(const esmm_grid *g, esmm_params *prm)
{
    if (!g || !prm) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_get_params(g->g3, prm);
    *prm = g->prm;
    return ESMM_OK;
}

int esmm_state_set(esmm_grid *g, const double *prim, const double *x, int mem)
{
    if (!g || !prim || g->nprob != 1) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_state_set(g->g3, prim, x, mem);
    if (g->nslab) {
        int rc = slab_state_set(g, prim, x, mem);
        g->has_state = rc == ESMM_OK;
        return rc;
    }
    int rc = state_set_one(g, 0, prim, x, mem);
    g->has_state = rc == ESMM_OK;
    return rc;
}

int esmm_state_set_cons(esmm_grid *g, const double *cons, const double *J, const double *x, double t, int mem)
{
    if (g && g->nslab) return fail(g, ESMM_ERR_ARG, "not available on a slab");
    if (!g || !cons || !J || !x || g->nprob != 1) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_state_set_cons(g->g3, cons, J, x, t, mem);
    size_t N = (size_t)g->Ntot, nv = (size_t)g->nv;
    int rc;
    if ((rc = copy_in(g, g->cons, cons, nv * N, mem)) || (rc = copy_in(g, g->J, J, N, mem)) ||
        (rc = copy_in(g, g->x, x, 2 * N, mem)))
        return rc;
    g->pin[0] = t;
    CK(cudaMemcpyAsync(g->t_dev, g->pin, sizeof(double), cudaMemcpyHostToDevice, g->st));
    CK(cudaMemsetAsync(g->xdot, 0, 2 * N * sizeof(double), g->st));
    for (int k = 0; k < 3; ++k) CK(cudaMemsetAsync(g->pg[k], 0xff, N * sizeof(double), g->st));
    CK(cudaStreamSynchronize(g->st));
    g->xdot_zero = 1;
    g->has_state = 1;
    return ESMM_OK;
}

int esmm_state_get(esmm_grid *g, int what, double *out, int mem)
{
    if (!g || !out || g->nprob != 1) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_state_get(g->g3, what, out, mem);
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    if (g->nslab) return slab_state_get(g, what, out, mem);
    return state_get_one(g, 0, what, out, mem);
}

int esmm_get_time(esmm_grid *g, double *t)
{
    if (!g || !t) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_get_time(g->g3, t);
    CK(cudaMemcpyAsync(g->pin, g->t_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    *t = g->pin[0];
    return ESMM_OK;
}

int esmm_rhs(esmm_grid *g, const double *cons, const double *J, const double *x, const double *xdot,
             double *dcons, double *dJ, int mem)
{
    if (!g || !cons || !J || !x || !dcons || !dJ || g->nprob != 1) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_rhs(g->g3, cons, J, x, xdot, dcons, dJ, mem);
    int rc;
    if ((rc = ensure_doms(g))) return rc;
    size_t N = (size_t)g->Ntot, nv = (size_t)g->nv;
    if (mem == ESMM_MEM_HOST) {
        if ((rc = copy_in(g, g->in_cons, cons, nv * N, mem)) || (rc = copy_in(g, g->in_J, J, N, mem)) ||
            (rc = copy_in(g, g->in_x, x, 2 * N, mem)))
            return rc;
        if (xdot && (rc = copy_in(g, g->in_xdot, xdot, 2 * N, mem))) return rc;
        cons = g->in_cons;
        J = g->in_J;
        x = g->in_x;
        xdot = xdot ? g->in_xdot : nullptr;
    }
    node(g, cons, J, x, xdot, nullptr, nullptr);
    fluxes(g);
    double *dc = mem == ESMM_MEM_HOST ? g->out_dc : dcons;
    double *dj = mem == ESMM_MEM_HOST ? g->out_dJ : dJ;
    update(g, dc, dj, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, 0.0, nullptr, nullptr,
           nullptr);
    CK(cudaGetLastError());
    if (mem == ESMM_MEM_HOST) {
        if ((rc = copy_out(g, dcons, g->out_dc, nv * N, mem)) || (rc = copy_out(g, dJ, g->out_dJ, N, mem)))
            return rc;
        CK(cudaStreamSynchronize(g->st));
        return check_c2p(g);
    }
    return ESMM_OK;
}

int esmm_cfl_dt(esmm_grid *g, double *dt)
{
    if (!g || !dt || g->nprob != 1) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_cfl_dt(g->g3, dt);
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    int rc;
    if ((rc = ensure_doms(g))) return rc;
    node(g, g->cons, g->J, g->x, nullptr, nullptr, nullptr);
    red_init(g);
    step_radius(g, 0.0, false);
    if (g->nslab && (rc = slab_slots(g, {2, 3}, {}))) return rc;   // the radius over every slab's own rows
    step_dt(g, 0.0, false);   // slots 4, 5 are zero: the static-mesh step
    CK(cudaMemcpyAsync(g->pin, g->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    *dt = g->pin[0];
    return check_c2p(g);
}

int esmm_mesh_redistribute(esmm_grid *g, double dt, double *xdot, double *dtau, double *dt_used, int mem)
{
    if (g && g->nslab) return fail(g, ESMM_ERR_ARG, "not available on a slab");
    if (!g || g->nprob != 1) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_mesh_redistribute(g->g3, dt, xdot, dtau, dt_used, mem);
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    int rc;
    if ((rc = ensure_doms(g))) return rc;
    node(g, g->cons, g->J, g->x, nullptr, nullptr, nullptr);
    red_init(g);
    step_radius(g, dt, g->prm.move_mesh);
    if ((rc = mesh_core(g, dt))) return rc;
    if (xdot && (rc = copy_out(g, xdot, g->xdot, 2 * (size_t)g->Ntot, mem))) return rc;
    CK(cudaMemcpyAsync(g->pin, g->red + 1, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaMemcpyAsync(g->pin + 1, g->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    if (dtau) *dtau = g->prm.move_mesh ? g->pin[0] : 0.0;
    if (dt_used) *dt_used = g->pin[1];
    return check_c2p(g);
}

int esmm_rk_step(esmm_grid *g, double dt, double *dt_used)
{
    if (!g) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_rk_step(g->g3, dt, dt_used);
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    int rc = g->nslab ? slab_step(g, dt) : rk_step_async(g, dt);
    if (rc) return rc;
    if (dt_used) {
        CK(cudaMemcpyAsync(g->pin, g->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, g->st));
        CK(cudaStreamSynchronize(g->st));
        *dt_used = g->pin[0];
        return check_c2p(g);
    }
    return ESMM_OK;
}

int esmm_rk_step_given(esmm_grid *g, const double *xdot, double dt, int mem)
{
    if (g && g->nslab) return fail(g, ESMM_ERR_ARG, "not available on a slab");
    if (!g || !xdot || !(dt > 0.0) || (mem != ESMM_MEM_HOST && mem != ESMM_MEM_DEVICE)) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_rk_step_given(g->g3, xdot, dt, mem);
    if (g->nprob != 1) return fail(g, ESMM_ERR_ARG, "a batch steps with its adaptive meshes");
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    int rc = step_given(g, xdot, dt, mem);
    if (rc) return rc;
    CK(cudaStreamSynchronize(g->st));
    return check_c2p(g);
}

int esmm_set_inflow(esmm_grid *g, const double *prim)
{
    if (g && g->nslab) return fail(g, ESMM_ERR_ARG, "not available on a slab");
    if (!g || !prim) return ESMM_ERR_ARG;
    const int nv = g->dim == 3 ? 8 : g->nv;
    double v2 = 0.0;
    for (int a = 1; a <= (nv == 8 ? 3 : 2); ++a) v2 += prim[a] * prim[a];
    const double p = prim[nv == 8 ? 4 : 3];
    if (!(prim[0] > 0.0) || !(p > 0.0) || !(v2 < 1.0)) return fail(g, ESMM_ERR_ARG, "inadmissible inflow state");
    if (g->dim == 3) return esmm3_set_inflow(g->g3, prim);
    double w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 0; a < nv; ++a) w[a] = prim[a];
    CK(cudaMemcpyAsync(g->inflow_dev, w, 8 * sizeof(double), cudaMemcpyHostToDevice, g->st));
    CK(cudaStreamSynchronize(g->st));
    g->has_inflow = 1;
    g->epoch++;
    return ESMM_OK;
}

int esmm_advance(esmm_grid *g, int nsteps, double dt)
{
    if (!g || nsteps < 0) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_advance(g->g3, nsteps, dt);
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    if (g->nslab) {   // no graph: every step reduces and exchanges through the host
        for (int k = 0; k < nsteps; ++k)
            if (int rc = slab_step(g, dt)) return rc;
        return ESMM_OK;
    }
    return advance(g, nsteps, dt);
}

int esmm_totals(esmm_grid *g, double out[3])
{
    if (!g || !out || g->nprob != 1) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_totals(g->g3, out);
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    int rc = totals_async(g);
    if (rc) return rc;
    CK(cudaMemcpyAsync(g->pin, g->tot_dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    for (int k = 0; k < 3; ++k) out[k] = g->pin[k];
    if (g->nslab && (rc = slab_allreduce(g, out, 3, ESMM_OP_SUM))) return rc;   // own rows of every slab
    return check_c2p(g);
}

// ---- batches -----------------------------------------------------------------
int esmm_batch_create(esmm_grid **out, int nprob, const int *n, const double *lo, const double *hi, const int *bc,
                      int phys, void *stream)
{
    if (!out || nprob < 1 || !n || !lo || !hi || !bc || phys != ESMM_RHD) return ESMM_ERR_ARG;
    *out = nullptr;
    for (int b = 0; b < nprob; ++b)
        if (check_geometry(n[2 * b], n[2 * b + 1], lo + 2 * b, hi + 2 * b, bc + 2 * b)) return ESMM_ERR_ARG;
    return create(out, nprob, n, lo, hi, bc, ESMM_RHD, stream, true);
}

int esmm_batch_size(const esmm_grid *g, int *nprob)
{
    if (g && g->dim == 3) return ESMM_ERR_ARG;   // RHD / 2D only
    if (!g || !nprob) return ESMM_ERR_ARG;
    *nprob = g->nprob;
    return ESMM_OK;
}

int esmm_batch_state_set(esmm_grid *g, int b, const double *prim, const double *x, int mem)
{
    if (g && g->dim == 3) return ESMM_ERR_ARG;   // RHD / 2D only
    if (!g || !prim || b < 0 || b >= g->nprob) return ESMM_ERR_ARG;
    int rc = state_set_one(g, b, prim, x, mem);
    if (rc == ESMM_OK) g->has_state = 1;
    return rc;
}

int esmm_batch_state_get(esmm_grid *g, int b, int what, double *out, int mem)
{
    if (g && g->dim == 3) return ESMM_ERR_ARG;   // RHD / 2D only
    if (!g || !out || b < 0 || b >= g->nprob) return ESMM_ERR_ARG;
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    return state_get_one(g, b, what, out, mem);
}

int esmm_batch_times(esmm_grid *g, double *t)
{
    if (g && g->dim == 3) return ESMM_ERR_ARG;   // RHD / 2D only
    if (!g || !t) return ESMM_ERR_ARG;
    CK(cudaMemcpyAsync(g->pin, g->t_dev, g->nprob * sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    for (int b = 0; b < g->nprob; ++b) t[b] = g->pin[b];
    return ESMM_OK;
}

int esmm_batch_totals(esmm_grid *g, double *out)
{
    if (g && g->dim == 3) return ESMM_ERR_ARG;   // RHD / 2D only
    if (!g || !out) return ESMM_ERR_ARG;
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    int rc = totals_async(g);
    if (rc) return rc;
    CK(cudaMemcpyAsync(g->pin, g->tot_dev, 3 * g->nprob * sizeof(double), cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    for (int k = 0; k < 3 * g->nprob; ++k) out[k] = g->pin[k];
    return check_c2p(g);
}

int esmm_tune(esmm_grid *g, int *block_sizes)
{
    if (g && g->nslab) return fail(g, ESMM_ERR_ARG, "not available on a slab");
    if (g && g->dim == 3) return ESMM_ERR_ARG;   // RHD / 2D only
    if (!g) return ESMM_ERR_ARG;
    int rc = tune(g);
    if (rc) return rc;
    if (block_sizes) {
        for (int k = 0; k < ND; ++k) block_sizes[k] = g->bs[k] * (g->order_lpt[k] ? -1 : 1);
        for (int k = 0; k < 4; ++k)   // tile shapes of the tiled pair / interface launches, x_1 then x_2
            block_sizes[ND + k] = g->tx[D_TPAIR0 + k] + (g->persist[D_TPAIR0 + k] ? 1000 : 0);
    }
    return ESMM_OK;
}

int esmm_rhs_vjp(esmm_grid *g, const double *cons, const double *J, const double *x, const double *xdot,
                 const double *mu, double *lam, int mem)
{
    if (g && g->nslab) return fail(g, ESMM_ERR_ARG, "not available on a slab");
    if (g && g->needs_inflow) return fail(g, ESMM_ERR_ARG, "the adjoint takes periodic and outflow ends");
    if (g && g->dim == 3) {
        if (!cons || !J || !x || !mu || !lam) return ESMM_ERR_ARG;
        return esmm3_rhs_vjp(g->g3, cons, J, x, xdot, mu, lam, mem);
    }
    if (!g || !cons || !J || !x || !mu || !lam || g->nprob != 1) return ESMM_ERR_ARG;
    if (g->phys == ESMM_RMHD && g->prm.precision != ESMM_FP64)
        return fail(g, ESMM_ERR_ARG, "the RMHD adjoint is FP64");
    int rc;
    if ((rc = ensure_doms(g)) || (rc = adj_alloc(g))) return rc;
    size_t N = (size_t)g->Ntot, nv = (size_t)g->nv;
    if (mem == ESMM_MEM_HOST) {
        if ((rc = copy_in(g, g->in_cons, cons, nv * N, mem)) || (rc = copy_in(g, g->in_J, J, N, mem)) ||
            (rc = copy_in(g, g->in_x, x, 2 * N, mem)) || (rc = copy_in(g, g->lam_a, mu, nv * N, mem)))
            return rc;
        if (xdot && (rc = copy_in(g, g->in_xdot, xdot, 2 * N, mem))) return rc;
        cons = g->in_cons;
        J = g->in_J;
        x = g->in_x;
        xdot = xdot ? g->in_xdot : nullptr;
        mu = g->lam_a;
    }
    double *out = mem == ESMM_MEM_HOST ? g->lam_v : lam;
    if ((rc = rhs_vjp_core(g, cons, J, x, xdot, mu, out))) return rc;
    if (mem == ESMM_MEM_HOST) {
        if ((rc = copy_out(g, lam, g->lam_v, nv * N, mem))) return rc;
        CK(cudaStreamSynchronize(g->st));
        return check_c2p(g);
    }
    return ESMM_OK;
}

int esmm_adjoint_record(esmm_grid *g, int nsteps, double dt)
{
    if (g && g->nslab) return fail(g, ESMM_ERR_ARG, "not available on a slab");
    if (g && g->needs_inflow) return fail(g, ESMM_ERR_ARG, "the adjoint takes periodic and outflow ends");
    if (g && g->dim == 3) return nsteps < 0 ? ESMM_ERR_ARG : esmm3_adjoint_record(g->g3, nsteps, dt);
    if (!g || nsteps < 0 || g->nprob != 1) return ESMM_ERR_ARG;
    if (g->phys == ESMM_RMHD && g->prm.precision != ESMM_FP64)
        return fail(g, ESMM_ERR_ARG, "the RMHD adjoint is FP64");
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    size_t N = (size_t)g->Ntot, d = sizeof(double), nv = (size_t)g->nv;
    g->ck_dt->clear();
    g->ck_n = 0;
    for (int n = 0; n < nsteps; ++n) {
        if ((int)g->ck->size() <= n) {
            double *b = nullptr;
            CK(cudaMalloc((void **)&b, (nv + 5) * N * d));   // cons, J, x, xdot
            g->ck->push_back(b);
        }
        double *b = (*g->ck)[n];
        CK(cudaMemcpyAsync(b, g->cons, nv * N * d, cudaMemcpyDeviceToDevice, g->st));
        CK(cudaMemcpyAsync(b + nv * N, g->J, N * d, cudaMemcpyDeviceToDevice, g->st));
        CK(cudaMemcpyAsync(b + (nv + 1) * N, g->x, 2 * N * d, cudaMemcpyDeviceToDevice, g->st));
        int rc = rk_step_async(g, dt);
        if (rc) return rc;
        CK(cudaMemcpyAsync(b + (nv + 3) * N, g->xdot, 2 * N * d, cudaMemcpyDeviceToDevice, g->st));
        CK(cudaMemcpyAsync(g->pin, g->dt_dev, d, cudaMemcpyDeviceToHost, g->st));
        CK(cudaStreamSynchronize(g->st));
        g->ck_dt->push_back(g->pin[0]);
        g->ck_n = n + 1;
    }
    return check_c2p(g);
}

int esmm_adjoint_steps(esmm_grid *g, int *nsteps, double *dt)
{
    if (g && g->dim == 3) return nsteps ? esmm3_adjoint_steps(g->g3, nsteps, dt) : ESMM_ERR_ARG;
    if (!g || !nsteps) return ESMM_ERR_ARG;
    *nsteps = g->ck_n;
    if (dt)
        for (int n = 0; n < g->ck_n; ++n) dt[n] = (*g->ck_dt)[n];
    return ESMM_OK;
}

int esmm_adjoint_checkpoint(esmm_grid *g, int step, int what, double *out, int mem)
{
    if (g && g->dim == 3) return out ? esmm3_adjoint_checkpoint(g->g3, step, what, out, mem) : ESMM_ERR_ARG;
    if (!g || !out || step < 0 || step >= g->ck_n) return ESMM_ERR_ARG;
    size_t N = (size_t)g->Ntot, nv = (size_t)g->nv;
    const double *b = (*g->ck)[step];
    int rc;
    switch (what) {
    case ESMM_GET_CONS: rc = copy_out(g, out, b, nv * N, mem); break;
    case ESMM_GET_J: rc = copy_out(g, out, b + nv * N, N, mem); break;
    case ESMM_GET_X: rc = copy_out(g, out, b + (nv + 1) * N, 2 * N, mem); break;
    case ESMM_GET_XDOT: rc = copy_out(g, out, b + (nv + 3) * N, 2 * N, mem); break;
    default: return fail(g, ESMM_ERR_ARG, "unknown field");
    }
    if (rc) return rc;
    CK(cudaStreamSynchronize(g->st));
    return ESMM_OK;
}

int esmm_adjoint_replay(esmm_grid *g, int nsteps)
{
    if (g && g->nslab) return fail(g, ESMM_ERR_ARG, "not available on a slab");
    if (g && g->dim == 3) return esmm3_adjoint_replay(g->g3, nsteps);
    if (!g || nsteps < 0 || nsteps > g->ck_n || g->nprob != 1) return ESMM_ERR_ARG;
    if (!g->has_state) return fail(g, ESMM_ERR_STATE, "no state");
    size_t N = (size_t)g->Ntot;
    for (int n = 0; n < nsteps; ++n) {
        int rc = step_given(g, (*g->ck)[n] + (g->nv + 3) * N, (*g->ck_dt)[n], ESMM_MEM_DEVICE);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(g->st));
    return check_c2p(g);
}

int esmm_adjoint_vjp(esmm_grid *g, const double *lam_final, double *lam_cons0, double *lam_prim0, int mem)
{
    if (g && g->nslab) return fail(g, ESMM_ERR_ARG, "not available on a slab");
    if (g && g->dim == 3) return lam_final ? esmm3_adjoint_vjp(g->g3, lam_final, lam_cons0, lam_prim0, mem)
                                           : ESMM_ERR_ARG;
    if (!g || !lam_final || g->nprob != 1) return ESMM_ERR_ARG;
    if (g->ck_n < 1) return fail(g, ESMM_ERR_STATE, "no recorded steps");
    int rc;
    if ((rc = ensure_doms(g)) || (rc = adj_alloc(g))) return rc;
    size_t N = (size_t)g->Ntot, nv = (size_t)g->nv;
    const long long n4 = (long long)(nv * N);
    double *la = g->lam_a, *lb = g->lam_b, *lc = g->lam_c, *v = g->lam_v;
    if ((rc = copy_in(g, la, lam_final, nv * N, mem))) return rc;
    for (int n = g->ck_n - 1; n >= 0; --n) {
        double *b = (*g->ck)[n];
        double *c0 = b, *J0 = b + nv * N, *x0 = b + (nv + 1) * N, *xd = b + (nv + 3) * N;
        double dt = (*g->ck_dt)[n];
        if ((rc = set_dt(g, dt))) return rc;
        // recompute the stage states (c1, J1, x1), (c2, J2, x2)
        node(g, c0, J0, x0, xd, nullptr, nullptr);
        fluxes(g);
        update(g, nullptr, nullptr, c0, J0, x0, c0, J0, x0, xd, 0.0, 1.0, g->c1, g->J1, g->x1);
        node(g, g->c1, g->J1, g->x1, xd, nullptr, nullptr);
        fluxes(g);
        update(g, nullptr, nullptr, c0, J0, x0, g->c1, g->J1, g->x1, xd, 0.75, 0.25, g->c2, g->J2, g->x2);
        // stage 3: c3 = 1/3 c0 + 2/3 (c2 + dt L(c2))
        if ((rc = rhs_vjp_core(g, g->c2, g->J2, g->x2, xd, la, v))) return rc;
        launch_lincomb(n4, 2.0 / 3.0, la, 2.0 / 3.0 * dt, v, lb, g->st);    // lambda_c2
        launch_lincomb(n4, 1.0 / 3.0, la, 0.0, nullptr, lc, g->st);         // lambda_c0
        // stage 2: c2 = 3/4 c0 + 1/4 (c1 + dt L(c1))
        if ((rc = rhs_vjp_core(g, g->c1, g->J1, g->x1, xd, lb, v))) return rc;
        launch_lincomb(n4, 0.25, lb, 0.25 * dt, v, la, g->st);              // lambda_c1
        launch_lincomb(n4, 1.0, lc, 0.75, lb, lc, g->st);
        // stage 1: c1 = c0 + dt L(c0)
        if ((rc = rhs_vjp_core(g, c0, J0, x0, xd, la, v))) return rc;
        launch_lincomb(n4, 1.0, lc, 1.0, la, lc, g->st);
        launch_lincomb(n4, 1.0, lc, dt, v, la, g->st);                      // lambda of c^n
    }
    CK(cudaGetLastError());
    if (lam_cons0 && (rc = copy_out(g, lam_cons0, la, nv * N, mem))) return rc;
    if (lam_prim0) {
        double *b0 = (*g->ck)[0];
        LaunchDom L = dom(g, D_NODE);
        if (g->phys == ESMM_RMHD) launch_prim_grad_mhd(L, g->gamma, b0, b0 + nv * N, la, v, g->status, g->st);
        else launch_prim_grad(L, g->gamma, b0, b0 + 4 * N, la, v, g->st);
        if ((rc = copy_out(g, lam_prim0, v, nv * N, mem))) return rc;
    }
    CK(cudaStreamSynchronize(g->st));
    return check_c2p(g);
}

int esmm_rhs_static(int nx, int ny, const int bc[2], const double lo[2], const double hi[2], double gamma, int p,
                    int w, const double *cons, const double *J, const double *x, const double *xdot, double *dcons,
                    double *dJ, void *stream)
{
    if (!bc || !lo || !hi || !cons || !J || !x || !dcons || !dJ) return ESMM_ERR_ARG;
    if (nx < 4 || ny < 4 || (long long)(nx + 2 * GH) * (ny + 2 * GH) > ESMM_STATIC_MAX_PADDED_NODES)
        return ESMM_ERR_ARG;
    for (int k = 0; k < 2; ++k)
        if ((bc[k] != ESMM_PERIODIC && bc[k] != ESMM_OUTFLOW) || !(hi[k] > lo[k])) return ESMM_ERR_ARG;
    if (!(gamma > 1.0 && gamma <= 2.0) || p < 1 || p > PMAX || !(w == 0 || w == 3 || w == 5)) return ESMM_ERR_ARG;
    // an error already pending on this thread is its owner's: leave it there
    // and enqueue nothing, so that no error of this call can be confused with it
    if (cudaPeekAtLastError() != cudaSuccess) return ESMM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    double *scratch = nullptr;
    if (static_scratch(st, &scratch) != cudaSuccess) {
        (void)cudaGetLastError();            // this call's own error (none was pending)
        return ESMM_ERR_CUDA;
    }
    ProbDesc D;
    Geom &G = D.g;
    G.nx = nx;
    G.ny = ny;
    G.px = nx + 2 * GH;
    G.py = ny + 2 * GH;
    G.P = (long long)G.px * G.py;
    G.N = (long long)nx * ny;
    G.bc0 = bc[0];
    G.bc1 = bc[1];
    G.own0 = 0;
    G.own1 = ny;
    G.per0 = hi[0] - lo[0];
    G.per1 = hi[1] - lo[1];
    D.on = 0;
    D.op = 0;
    Phys ph;
    ph.gamma = gamma;
    ph.eps = 1e-6;
    ph.gm1i = 1.0 / (gamma - 1.0);
    ph.ln_thr = 1.0e-4;
    ph.sign_tol = 1.0e-10;
    double a[3][3] = {{1.0, 0.0, 0.0}, {4.0 / 3.0, -1.0 / 6.0, 0.0}, {1.5, -0.3, 1.0 / 30.0}};
    for (int n = 0; n < PMAX; ++n) ph.alpha[n] = a[p - 1][n];
    ph.p = p;
    ph.w = w;
    // carve the scratch: node arrays, pair fluxes, interface fluxes, status
    double *q = scratch;
    double *pairs = q + (long long)NQ * G.P;
    double *iflux = pairs + (long long)2 * PMAX * 4 * G.P;
    int *status = (int *)(scratch + STATIC_PER_NODE * ESMM_STATIC_MAX_PADDED_NODES);
    if (cudaMemsetAsync(status, 0, 2 * sizeof(int), st) != cudaSuccess) {
        (void)cudaGetLastError();
        return ESMM_ERR_CUDA;
    }
    auto one = [&](long long count, int bs) {
        LaunchDom L;
        L.pa.pd = nullptr;
        L.pa.tiles = nullptr;
        L.pa.one = D;
        L.bs = bs;
        L.nblk = (unsigned)((count + bs - 1) / bs);
        return L;
    };
    LaunchDom Ln = one(G.P, BS);
    const double gg = (gamma - 1.0) / gamma;
    if (p == 1)
        k_node<1><<<Ln.nblk, Ln.bs, 0, st>>>(Ln.pa, gamma, gg, cons, J, x, xdot, nullptr, nullptr, q, status,
                                             nullptr, nullptr);
    else if (p == 2)
        k_node<2><<<Ln.nblk, Ln.bs, 0, st>>>(Ln.pa, gamma, gg, cons, J, x, xdot, nullptr, nullptr, q, status,
                                             nullptr, nullptr);
    else
        k_node<3><<<Ln.nblk, Ln.bs, 0, st>>>(Ln.pa, gamma, gg, cons, J, x, xdot, nullptr, nullptr, q, status,
                                             nullptr, nullptr);
    for (int dir = 0; dir < 2; ++dir) {
        long long cp = dir == 0 ? (long long)(nx + p) * ny : (long long)(ny + p) * nx;
        long long ci = dir == 0 ? (long long)(nx + 1) * ny : (long long)(ny + 1) * nx;
        launch_pairs_f64(one(cp, 128), ph, q, nullptr, pairs, dir, st);
        launch_iface_f64(one(ci, 128), ph, q, nullptr, pairs, iflux, dir, st);
    }
    LaunchDom Lu = one(G.N, BS);
    k_update<double><<<Lu.nblk, Lu.bs, 0, st>>>(Lu.pa, iflux, dcons, dJ, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                nullptr, nullptr, 0.0, 0.0, nullptr, nullptr, nullptr, nullptr);
    // nothing was pending on entry, so an error now is this call's own launch
    // error: consume it and report it
    if (cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();
        return ESMM_ERR_CUDA;
    }
    return ESMM_OK;
}

int esmm_profile(esmm_grid *g, int mask)
{
    if (!g || mask < 0 || mask >= (1 << ESMM_NKINDS)) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_profile(g->g3, mask);
    CK(cudaStreamSynchronize(g->st));
    for (int k = 0; k < ESMM_NKINDS; ++k) {
        for (auto &pr : g->ev[k]) { g->pool->push_back(pr.first); g->pool->push_back(pr.second); }
        g->ev[k].clear();
        g->launches[k] = 0;
        g->gms[k] = 0.0;
        g->gtimed[k] = 0;
    }
    g->gev_pending = 0;   // a finished replay's graph events are dropped with the counters
    g->prof_mask = mask;
    return ESMM_OK;
}

int esmm_profile_read(esmm_grid *g, double ms[ESMM_NKINDS], long long launches[ESMM_NKINDS],
                      long long timed[ESMM_NKINDS])
{
    if (!g) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_profile_read(g->g3, ms, launches, timed);
    CK(cudaStreamSynchronize(g->st));
    int rc = collect_graph_prof(g);
    if (rc) return rc;
    for (int k = 0; k < ESMM_NKINDS; ++k) {
        double acc = g->gms[k];
        for (auto &pr : g->ev[k]) {
            float t = 0.0f;
            CK(cudaEventElapsedTime(&t, pr.first, pr.second));
            acc += t;
        }
        if (ms) ms[k] = acc;
        if (launches) launches[k] = g->launches[k];
        if (timed) timed[k] = (long long)g->ev[k].size() + g->gtimed[k];
    }
    return ESMM_OK;
}

int esmm_last_error(esmm_grid *g, int *n_c2p_fail, char *msg, int len)
{
    if (!g) return ESMM_ERR_ARG;
    if (g->dim == 3) return esmm3_last_error(g->g3, n_c2p_fail, msg, len);
    int h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, g->status, sizeof h, cudaMemcpyDeviceToHost, g->st));
    CK(cudaStreamSynchronize(g->st));
    CK(cudaMemsetAsync(g->status, 0, sizeof(int), g->st));
    CK(cudaStreamSynchronize(g->st));
    if (n_c2p_fail) *n_c2p_fail = h[0];
    if (msg && len > 0) {
        strncpy(msg, g->msg, (size_t)len - 1);
        msg[len - 1] = '\0';
    }
    return ESMM_OK;
}

}  // extern "C"
