// esmm_flux.cuh -- the two flux kernels of one sweep direction:
//   k_pairs: every two-point EC flux F~_k(U_A, U_{A+n}) (Sec. 3.1), n = 1..p,
//            computed once per node pair and stored;
//   k_iface: the w-th order ES interface flux (eq. ESFlux_HO): the 2p-th order
//            combination of the stored pair fluxes (eq. ECFlux_O2p) minus the
//            WENO dissipation on scaled entropy variables, plus the metric
//            flux of the VCL (eq. MetricsFlux_O2p).
// One thread per node pair / interface, flattened over the sweep so that warps
// read consecutive nodes.
#pragma once

#include <type_traits>

#include "esmm_device.cuh"
#include "esmm_launch.h"

namespace esmm {

// One flux argument: the FP64 log-mean arguments from q and the working
// values from q (FP64) or from the FP32 copies q32 (float).
template <typename R>
__device__ __forceinline__ NodeV<R> load_node(const Geom &g, const double *__restrict__ q,
                                              const float *__restrict__ q32, long long c)
{
    NodeV<R> v;
    v.rho = q[Q_RHO * g.P + c];
    v.beta = q[Q_BETA * g.P + c];
    v.lnr = q[Q_LNR * g.P + c];
    v.lnb = q[Q_LNB * g.P + c];
    if constexpr (std::is_same<R, float>::value) {
        v.r = q32[Q32_R * g.P + c];
        v.b = q32[Q32_B * g.P + c];
        v.ux = q32[Q32_UX * g.P + c];
        v.uy = q32[Q32_UY * g.P + c];
        v.W = q32[Q32_W * g.P + c];
    } else {
        v.r = (R)v.rho;
        v.b = (R)v.beta;
        v.ux = (R)q[Q_UX * g.P + c];
        v.uy = (R)q[Q_UY * g.P + c];
        v.W = (R)q[Q_W * g.P + c];
    }
    return v;
}

// The ES dissipation 1/2 lambda^ T^-1 R Y <<V~>> of eq. ESFlux_HO at one
// interface (to be subtracted from the EC flux).  nvx, nvy, jt: the interface
// metrics (mean of the two nodes); rho0/1, lnr0/1: density and its log at the
// two interface nodes (the log-mean arguments), r0/1 the densities in the
// working precision; st[k] = (beta, u_x, u_y, W,
// ln rho, ln beta) of the w + 1 stencil nodes, the interface nodes at
// k = (w-1)/2 and (w+1)/2.  The eigen-system is taken at rho = {{rho}}^ln,
// u = {{u}}, p = {{rho}}/{{beta}}; Y has sign 0 for jumps at rounding level.
// The entropy variables (V_1, V_x, V_y, V_E) of one node (Sec. 2, B = 0)
// from beta, u, W, ln rho, ln beta: V_1 = Gamma/(Gamma-1) + ln rho +
// ln beta/(Gamma-1) + beta, (V_x, V_y) = beta u, V_E = -beta W.  Every
// stencil type below forms them with this one function, so a kernel that
// stores them per node gets the values a kernel forming them per interface
// gets: in FP64 and FP32 each operation is an explicitly rounded intrinsic,
// which leaves the compiler no choice of contraction between the two.
template <typename R>
__device__ __forceinline__ void entropy_vars4(R b, R ux, R uy, R W, R lnr, R lnb, R c1g, R ig, R V[4])
{
    V[0] = c1g + lnr + ig * lnb + b;
    V[1] = b * ux;
    V[2] = b * uy;
    V[3] = -b * W;
}
template <>
__device__ __forceinline__ void entropy_vars4<double>(double b, double ux, double uy, double W, double lnr,
                                                      double lnb, double c1g, double ig, double V[4])
{
    V[0] = __dadd_rn(__fma_rn(ig, lnb, __dadd_rn(c1g, lnr)), b);
    V[1] = __dmul_rn(b, ux);
    V[2] = __dmul_rn(b, uy);
    V[3] = -__dmul_rn(b, W);
}
template <>
__device__ __forceinline__ void entropy_vars4<float>(float b, float ux, float uy, float W, float lnr, float lnb,
                                                     float c1g, float ig, float V[4])
{
    V[0] = __fadd_rn(__fmaf_rn(ig, lnb, __fadd_rn(c1g, lnr)), b);
    V[1] = __fmul_rn(b, ux);
    V[2] = __fmul_rn(b, uy);
    V[3] = -__fmul_rn(b, W);
}

// stencil values read straight from the node arrays (forward kernels)
template <typename R>
struct QStencil {
    const double *q;
    long long P, c0, sd;
    int off;
    __device__ __forceinline__ R operator()(int k, int j) const
    {
        const int f = j == 0 ? Q_BETA : (j == 1 ? Q_UX : (j == 2 ? Q_UY : (j == 3 ? Q_W : (j == 4 ? Q_LNR : Q_LNB))));
        return (R)q[f * P + c0 + (k - off) * sd];
    }
    __device__ __forceinline__ void V(int k, R c1g, R ig, R v[4]) const
    {
        entropy_vars4<R>((*this)(k, 0), (*this)(k, 1), (*this)(k, 2), (*this)(k, 3), (*this)(k, 4), (*this)(k, 5), c1g,
                         ig, v);
    }
};

// the same from the FP32 copies (the mixed form)
struct QStencil32 {
    const float *q;
    long long P, c0, sd;
    int off;
    __device__ __forceinline__ float operator()(int k, int j) const
    {
        const int f = j == 0 ? Q32_B
                    : (j == 1 ? Q32_UX : (j == 2 ? Q32_UY : (j == 3 ? Q32_W : (j == 4 ? Q32_LNR : Q32_LNB))));
        return q[f * P + c0 + (k - off) * sd];
    }
    __device__ __forceinline__ void V(int k, float c1g, float ig, float v[4]) const
    {
        entropy_vars4<float>((*this)(k, 0), (*this)(k, 1), (*this)(k, 2), (*this)(k, 3), (*this)(k, 4), (*this)(k, 5),
                             c1g, ig, v);
    }
};

// stencil values held in an array (the adjoint's seeded duals)
template <typename R, int NS>
struct ArrStencil {
    const R (*a)[6];
    __device__ __forceinline__ R operator()(int k, int j) const { return a[k][j]; }
    __device__ __forceinline__ void V(int k, R c1g, R ig, R v[4]) const
    {
        entropy_vars4<R>(a[k][0], a[k][1], a[k][2], a[k][3], a[k][4], a[k][5], c1g, ig, v);
    }
};

template <typename R, typename T, int WW, typename ST>
__device__ __forceinline__ void es_dissipation(R nvx, R nvy, R jt, T rho0, T rho1, T lnr0, T lnr1, R r0, R r1,
                                               const ST &st, const Phys &ph, R diss[4])
{
    constexpr int NS = WW + 1, OFF = (WW - 1) / 2;
    const R half = (R)0.5, one = (R)1;
    const R gam = (R)ph.gamma;
    R n2 = nvx * nvx + nvy * nvy;
    R iLk = rsq<R>(n2);
    R Lk = n2 * iLk;
    R nx = nvx * iLk, ny = nvy * iLk;
    R rho, irho;
    lmean<R, T>(rho0, rho1, lnr0, lnr1, r0, r1, ph.ln_thr, rho, irho);
    R ux = half * (st(OFF, 1) + st(OFF + 1, 1));
    R uy = half * (st(OFF, 2) + st(OFF + 1, 2));
    R p = (r0 + r1) * rcp<R>(st(OFF, 0) + st(OFF + 1, 0));
    R w2 = one + ux * ux + uy * uy;
    R iW = rsq<R>(w2);
    R W = w2 * iW;
    R vx = ux * iW, vy = uy * iW;
    R vn = nx * vx + ny * vy, vt = -ny * vx + nx * vy;
    R dU[4][4], s[4], lm, lp;
    const R ig = (R)ph.gm1i, c1g = gam * ig;
    eigen_rhd<R>(gam, ig, rho, vn, vt, p, W, dU, s, lm, lp);
    R lhat = vmax(fab<R>(jt + Lk * lm), fab<R>(jt + Lk * lp));
    // Vt_m = s_m dU_m . (T V): the rotation T and the scale s_m folded into
    // the projection row Ar[m] once per interface
    R Ar[4][4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        Ar[m][0] = s[m] * dU[0][m];
        Ar[m][1] = s[m] * (nx * dU[1][m] - ny * dU[2][m]);
        Ar[m][2] = s[m] * (ny * dU[1][m] + nx * dU[2][m]);
        Ar[m][3] = s[m] * dU[3][m];
    }
    R Vt[NS][4];
    R aT[4] = {(R)0, (R)0, (R)0, (R)0};     // |T V| summed over the two interface nodes
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        R V[4];
        st.V(k, c1g, ig, V);
        if (k == OFF || k == OFF + 1) {
            aT[0] += fab<R>(V[0]);
            aT[1] += fab<R>(nx * V[1] + ny * V[2]);
            aT[2] += fab<R>(-ny * V[1] + nx * V[2]);
            aT[3] += fab<R>(V[3]);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) Vt[k][m] = Ar[m][0] * V[0] + Ar[m][1] * V[1] + Ar[m][2] * V[2] + Ar[m][3] * V[3];
    }
    const R eps = (R)ph.eps;
    const R sign_tol = (R)ph.sign_tol;
    R z[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        R vminus, vplus;
        if (WW == 5)
            weno5_lr<R>(Vt[0][m], Vt[1][m], Vt[2][m], Vt[3][m], Vt[4][m], Vt[5][m], eps, vminus, vplus);
        else
            weno3_lr<R>(Vt[0][m], Vt[1][m], Vt[2][m], Vt[3][m], eps, vminus, vplus);
        R jw = vplus - vminus;
        R jump = Vt[OFF + 1][m] - Vt[OFF][m];
        // a jump within sign_tol of the magnitudes forming V~_m at the two
        // interface nodes is rounding noise: its sign is 0 (so Y = 0)
        R scale = s[m] * (fab<R>(dU[0][m]) * aT[0] + fab<R>(dU[1][m]) * aT[1] +
                          fab<R>(dU[2][m]) * aT[2] + fab<R>(dU[3][m]) * aT[3]);
        int sj = le(fab<R>(jump), sign_tol * scale) ? 0 : sgn_d(jump);
        z[m] = (sgn_d(jw) == sj) ? jw * s[m] : (R)0;
    }
    R d[4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
        d[a] = dU[a][0] * z[0] + dU[a][1] * z[1] + dU[a][2] * z[2] + dU[a][3] * z[3];
    R hl = half * lhat;
    diss[0] = hl * d[0];
    diss[1] = hl * (nx * d[1] - ny * d[2]);
    diss[2] = hl * (ny * d[1] + nx * d[2]);
    diss[3] = hl * d[3];
}

// anchors A in [-P, n_dir - 1] along the sweep, every line of the other
// index: the sites of tile t (sweep_site)
template <typename R, int P>
__device__ __forceinline__ void pairs_tile(const ProbArg &pa, const Phys &ph, const double *__restrict__ q,
                                           const float *__restrict__ q32, R *__restrict__ pairs, int dir, int tx,
                                           long long t)
{
    constexpr bool F32 = std::is_same<R, float>::value;
    ProbDesc D;
    long long lb;
    locate_tile(pa, t, D, lb);
    const Geom &g = D.g;
    q += (long long)NQ * D.op;
    if (F32) q32 += (long long)NQ32 * D.op;
    pairs += (long long)2 * PMAX * 4 * D.op;
    int i, j;
    if (!sweep_site(g, dir, P, tx, lb, i, j)) return;
    const long long c0 = pidx(g, i, j);
    const long long sd = dir == 0 ? 1 : g.px;
    // metrics in the working precision: FP64 node arrays or their FP32 copies
    using MT = typename std::conditional<F32, float, double>::type;
    const MT *Mt, *Mx, *My;
    if constexpr (F32) {
        Mt = q32 + (Q32_MT0 + dir) * g.P;
        Mx = q32 + (Q32_M00 + 2 * dir) * g.P;
        My = q32 + (Q32_M01 + 2 * dir) * g.P;
    } else {
        Mt = q + (Q_MT0 + dir) * g.P;
        Mx = q + (Q_M00 + 2 * dir) * g.P;
        My = q + (Q_M01 + 2 * dir) * g.P;
    }
    const R gm1inv = (R)(1.0 / (ph.gamma - 1.0));
    NodeV<R> l = load_node<R>(g, q, q32, c0);
    const MT mtl = Mt[c0], mxl = Mx[c0], myl = My[c0];
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        const long long cr = c0 + n * sd;
        NodeV<R> r = load_node<R>(g, q, q32, cr);
        R mt = (R)((MT)0.5 * (mtl + Mt[cr]));
        R mx = (R)((MT)0.5 * (mxl + Mx[cr]));
        R my = (R)((MT)0.5 * (myl + My[cr]));
        R out[4];
        ec_pair<R>(l, r, mt, mx, my, gm1inv, ph.ln_thr, out);
#pragma unroll
        for (int a = 0; a < 4; ++a)
            pairs[((long long)((dir * PMAX + (n - 1)) * 4 + a)) * g.P + c0] = out[a];
    }
}

// the blocks stride over the ntiles tiles (one tile each when the grid has
// ntiles blocks; a persistent grid when it has fewer)
template <typename R, int P>
__global__ void __launch_bounds__(128) k_pairs(ProbArg pa, Phys ph, const double *__restrict__ q,
                                               const float *__restrict__ q32, R *__restrict__ pairs, int dir, int tx,
                                               long long ntiles)
{
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) pairs_tile<R, P>(pa, ph, q, q32, pairs, dir, tx, t);
}

// interfaces between left node L in [-1, n_dir - 1] and L + 1: the sites of
// tile t (sweep_site)
template <typename R, int P, int WW>
__device__ __forceinline__ void iface_tile(const ProbArg &pa, const Phys &ph, const double *__restrict__ q,
                                           const float *__restrict__ q32, const R *__restrict__ pairs,
                                           R *__restrict__ iflux, int dir, int tx, long long t)
{
    constexpr bool F32 = std::is_same<R, float>::value;
    using MT = typename std::conditional<F32, float, double>::type;
    ProbDesc D;
    long long lb;
    locate_tile(pa, t, D, lb);
    const Geom &g = D.g;
    q += (long long)NQ * D.op;
    if (F32) q32 += (long long)NQ32 * D.op;
    pairs += (long long)2 * PMAX * 4 * D.op;
    iflux += (long long)2 * 5 * D.op;
    int i, j;
    if (!sweep_site(g, dir, 1, tx, lb, i, j)) return;
    const long long c0 = pidx(g, i, j);
    const long long sd = dir == 0 ? 1 : g.px;
    // metrics in the working precision: FP64 node arrays or their FP32 copies
    const MT *Mt, *Mx, *My;
    if constexpr (F32) {
        Mt = q32 + (Q32_MT0 + dir) * g.P;
        Mx = q32 + (Q32_M00 + 2 * dir) * g.P;
        My = q32 + (Q32_M01 + 2 * dir) * g.P;
    } else {
        Mt = q + (Q_MT0 + dir) * g.P;
        Mx = q + (Q_M00 + 2 * dir) * g.P;
        My = q + (Q_M01 + 2 * dir) * g.P;
    }

    // eq. ECFlux_O2p: sum_n alpha_{p,n} sum_{s<n} F~(A - s, A - s + n)
    R F[4] = {(R)0, (R)0, (R)0, (R)0};
    MT Ft = (MT)0;
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        R Fs[4] = {(R)0, (R)0, (R)0, (R)0};
        MT Fts = (MT)0;
#pragma unroll
        for (int s = 0; s < n; ++s) {
            const long long ca = c0 - s * sd;
            const R *pr = pairs + ((long long)(dir * PMAX + (n - 1)) * 4) * g.P + ca;
#pragma unroll
            for (int a = 0; a < 4; ++a) Fs[a] += pr[a * g.P];
            Fts += (MT)0.5 * (Mt[ca] + Mt[ca + n * sd]);
        }
        const R an = (R)ph.alpha[n - 1];
#pragma unroll
        for (int a = 0; a < 4; ++a) F[a] += an * Fs[a];
        Ft += (MT)ph.alpha[n - 1] * Fts;
    }

    if (WW > 0) {
        // eq. ESFlux_HO: subtract 1/2 lambda^ T^-1 R Y <<V~>>
        const long long c1 = c0 + sd;
        const R nvx = (R)((MT)0.5 * (Mx[c0] + Mx[c1])), nvy = (R)((MT)0.5 * (My[c0] + My[c1]));
        const R jt = (R)((MT)0.5 * (Mt[c0] + Mt[c1]));
        const double rho0 = q[Q_RHO * g.P + c0], rho1 = q[Q_RHO * g.P + c1];
        const double lnr0 = q[Q_LNR * g.P + c0], lnr1 = q[Q_LNR * g.P + c1];
        R diss[4];
        if constexpr (F32) {
            QStencil32 st{q32, g.P, c0, sd, (WW - 1) / 2};
            es_dissipation<R, double, WW>(nvx, nvy, jt, rho0, rho1, lnr0, lnr1, q32[Q32_R * g.P + c0],
                                          q32[Q32_R * g.P + c1], st, ph, diss);
        } else {
            QStencil<R> st{q, g.P, c0, sd, (WW - 1) / 2};
            es_dissipation<R, double, WW>(nvx, nvy, jt, rho0, rho1, lnr0, lnr1, (R)rho0, (R)rho1, st, ph, diss);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) F[a] -= diss[a];
    }
    R *out = iflux + (long long)(dir * 5) * g.P + c0;
#pragma unroll
    for (int a = 0; a < 4; ++a) out[a * g.P] = F[a];
    out[4 * g.P] = (R)Ft;
}

template <typename R, int P, int WW>
__global__ void __launch_bounds__(128) k_iface(ProbArg pa, Phys ph, const double *__restrict__ q,
                                               const float *__restrict__ q32, const R *__restrict__ pairs,
                                               R *__restrict__ iflux, int dir, int tx, long long ntiles)
{
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x)
        iface_tile<R, P, WW>(pa, ph, q, q32, pairs, iflux, dir, tx, t);
}

inline long long tiles_of(const LaunchDom &L) { return L.ntiles < 0 ? (long long)L.nblk : L.ntiles; }

template <typename R, int P>
static void launch_pairs_p(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, R *pairs, int dir,
                           cudaStream_t st)
{
    k_pairs<R, P><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, q32, pairs, dir, L.tx, tiles_of(L));
}

template <typename R, int P, int WW>
static void launch_iface_pw(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, const R *pairs,
                            R *iflux, int dir, cudaStream_t st)
{
    k_iface<R, P, WW><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, q32, pairs, iflux, dir, L.tx, tiles_of(L));
}

// resident blocks per SM of one instance at block size bs
template <typename K>
static int occ(K kern, int bs)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, bs, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

template <typename R>
int flux_occupancy_t(int kind, int p, int w, int bs)
{
    if (kind == 0) return p == 1 ? occ(k_pairs<R, 1>, bs) : (p == 2 ? occ(k_pairs<R, 2>, bs) : occ(k_pairs<R, 3>, bs));
    auto pick = [&](auto k0, auto k3, auto k5) { return w == 0 ? occ(k0, bs) : (w == 3 ? occ(k3, bs) : occ(k5, bs)); };
    if (p == 1) return pick(k_iface<R, 1, 0>, k_iface<R, 1, 3>, k_iface<R, 1, 5>);
    if (p == 2) return pick(k_iface<R, 2, 0>, k_iface<R, 2, 3>, k_iface<R, 2, 5>);
    return pick(k_iface<R, 3, 0>, k_iface<R, 3, 3>, k_iface<R, 3, 5>);
}

template <typename R>
void launch_pairs_t(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, void *pairs, int dir,
                    cudaStream_t st)
{
    R *pr = (R *)pairs;
    switch (ph.p) {
    case 1: launch_pairs_p<R, 1>(L, ph, q, q32, pr, dir, st); break;
    case 2: launch_pairs_p<R, 2>(L, ph, q, q32, pr, dir, st); break;
    default: launch_pairs_p<R, 3>(L, ph, q, q32, pr, dir, st); break;
    }
}

template <typename R, int P>
static void launch_iface_p(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, const R *pr, R *fl,
                           int dir, cudaStream_t st)
{
    switch (ph.w) {
    case 0: launch_iface_pw<R, P, 0>(L, ph, q, q32, pr, fl, dir, st); break;
    case 3: launch_iface_pw<R, P, 3>(L, ph, q, q32, pr, fl, dir, st); break;
    default: launch_iface_pw<R, P, 5>(L, ph, q, q32, pr, fl, dir, st); break;
    }
}

template <typename R>
void launch_iface_t(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, const void *pairs,
                    void *iflux, int dir, cudaStream_t st)
{
    const R *pr = (const R *)pairs;
    R *fl = (R *)iflux;
    switch (ph.p) {
    case 1: launch_iface_p<R, 1>(L, ph, q, q32, pr, fl, dir, st); break;
    case 2: launch_iface_p<R, 2>(L, ph, q, q32, pr, fl, dir, st); break;
    default: launch_iface_p<R, 3>(L, ph, q, q32, pr, fl, dir, st); break;
    }
}

}  // namespace esmm
