// esmm_sweep.cuh -- the fused sweep kernel of one direction (2D RHD): the
// two-point EC fluxes (Sec. 3.1) and the ES interface fluxes (eq. ESFlux_HO)
// in one launch, with the node data of each tile and its pair fluxes held
// in shared memory.
//
// A warp owns one grid line (a row for the x_1 sweep, a column for the x_2
// sweep) and a segment of TA = 33 - p consecutive interfaces on it: its 32
// lanes first evaluate the 32 anchors A = L0 - (p - 1) .. L0 + 31 - (p - 1)
// (each anchor's p pair fluxes F~(A, A + n), as k_pairs does), store them in
// shared memory, and then the first TA lanes combine them into the
// interfaces L0 .. L0 + TA - 1 (eq. ECFlux_O2p) and subtract the WENO
// dissipation read from the staged stencil, as k_iface does.  The arithmetic
// is the same device code in the same order, so the interface fluxes equal
// those of the two-kernel path bit for bit; what changes is that the pair
// fluxes never leave the SM and every node value is read from global memory
// once per tile.
//
// Staging: the segment's nodes L0 - HL .. L0 + TA - 1 + HR (HL, HR the reach
// of the pairs and of the WENO stencil) for NW = blockDim.x / 32 lines.  In
// the x_1 sweep each warp reads its own row segment (consecutive addresses);
// in the x_2 sweep the block reads the NW columns row by row (NW consecutive
// addresses per row) and each warp then walks its column.  Per-warp arrays
// are laid out [field][node] with a stride of 41 nodes (conflict-free for
// both the row reads of the lanes and the column-interleaved staging writes).
// The staging also forms each node's entropy variables once (entropy_vars4,
// the rounded operations the two-kernel path applies per interface), which
// the dissipation then reads for every stencil that holds the node.
#pragma once

#include <type_traits>

#include "esmm_flux.cuh"

namespace esmm {

constexpr int SW_NNP = 41;   // node stride of a staged field (>= the largest segment, 37 nodes)

template <typename R, int P>
struct SweepLayout {
    static constexpr bool F32 = std::is_same<R, float>::value;
    // FP64 fields: rho, beta, ln rho, ln beta (the log-mean arguments), and in
    // the FP64 form also u_x, u_y, W, the direction's metrics Mt, Mx, My and
    // the entropy variables V_1, V_x, V_y, V_E
    static constexpr int NF64 = F32 ? 4 : 14;
    // FP32 fields of the mixed form: r, b, u_x, u_y, W, ln rho, ln beta, Mt,
    // Mx, My, V_1, V_x, V_y, V_E
    static constexpr int NF32 = F32 ? 14 : 0;
    static constexpr int PAIR_VALUES = P * 4 * 32;   // pair fluxes of the warp's 32 anchors
    static constexpr size_t bytes_per_warp =
        (size_t)NF64 * SW_NNP * 8 + (size_t)NF32 * SW_NNP * 4 + (size_t)PAIR_VALUES * sizeof(R);
};

template <int P, int WW>
struct SweepShape {
    static constexpr int HL = (P - 1 > (WW - 1) / 2) ? P - 1 : (WW - 1) / 2;
    static constexpr int HR = (P > (WW + 1) / 2) ? P : (WW + 1) / 2;
    static constexpr int TA = 33 - P;
    static_assert(TA + HL + HR <= SW_NNP, "segment exceeds the staged node stride");
};

// the staged stencil of es_dissipation: field j of node k (k = 0 .. WW)
template <typename R>
struct SmemStencil;
template <>
struct SmemStencil<double> {
    const double *s;
    int base;
    __device__ __forceinline__ double operator()(int k, int j) const
    {
        const int f = j == 0 ? 1 : (j == 1 ? 4 : (j == 2 ? 5 : (j == 3 ? 6 : (j == 4 ? 2 : 3))));
        return s[f * SW_NNP + base + k];
    }
    // the entropy variables staged with the node (fields 10 .. 13)
    __device__ __forceinline__ void V(int k, double, double, double v[4]) const
    {
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] = s[(10 + a) * SW_NNP + base + k];
    }
};
template <>
struct SmemStencil<float> {
    const float *s;
    int base;
    __device__ __forceinline__ float operator()(int k, int j) const
    {
        const int f = j == 0 ? 1 : (j == 1 ? 2 : (j == 2 ? 3 : (j == 3 ? 4 : (j == 4 ? 5 : 6))));
        return s[f * SW_NNP + base + k];
    }
    __device__ __forceinline__ void V(int k, float, float, float v[4]) const
    {
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] = s[(10 + a) * SW_NNP + base + k];
    }
};

// one node of global padded index c into staged slot e of a warp's arrays,
// with its entropy variables (entropy_vars4 on the staged values, as the
// stencils of the two-kernel path form them per interface)
template <typename R>
__device__ __forceinline__ void sweep_stage(const Geom &g, const double *__restrict__ q,
                                            const float *__restrict__ q32, long long c, int dir, R c1g, R ig,
                                            double *sd, float *sf, int e)
{
    if constexpr (std::is_same<R, float>::value) {
        sd[0 * SW_NNP + e] = q[Q_RHO * g.P + c];
        sd[1 * SW_NNP + e] = q[Q_BETA * g.P + c];
        sd[2 * SW_NNP + e] = q[Q_LNR * g.P + c];
        sd[3 * SW_NNP + e] = q[Q_LNB * g.P + c];
        const int fl[10] = {Q32_R, Q32_B, Q32_UX, Q32_UY, Q32_W, Q32_LNR, Q32_LNB, Q32_MT0 + dir, Q32_M00 + 2 * dir,
                            Q32_M01 + 2 * dir};
        float v[10];
#pragma unroll
        for (int f = 0; f < 10; ++f) sf[f * SW_NNP + e] = v[f] = q32[fl[f] * g.P + c];
        float V[4];
        entropy_vars4<float>(v[1], v[2], v[3], v[4], v[5], v[6], c1g, ig, V);
#pragma unroll
        for (int a = 0; a < 4; ++a) sf[(10 + a) * SW_NNP + e] = V[a];
    } else {
        const int fl[10] = {Q_RHO, Q_BETA, Q_LNR, Q_LNB, Q_UX, Q_UY, Q_W, Q_MT0 + dir, Q_M00 + 2 * dir,
                            Q_M01 + 2 * dir};
        double v[10];
#pragma unroll
        for (int f = 0; f < 10; ++f) sd[f * SW_NNP + e] = v[f] = q[fl[f] * g.P + c];
        double V[4];
        entropy_vars4<double>(v[1], v[4], v[5], v[6], v[2], v[3], c1g, ig, V);
#pragma unroll
        for (int a = 0; a < 4; ++a) sd[(10 + a) * SW_NNP + e] = V[a];
    }
}

// NodeV of staged slot i (as load_node)
template <typename R>
__device__ __forceinline__ NodeV<R> sweep_node(const double *sd, const float *sf, int i)
{
    NodeV<R> v;
    v.rho = sd[0 * SW_NNP + i];
    v.beta = sd[1 * SW_NNP + i];
    v.lnr = sd[2 * SW_NNP + i];
    v.lnb = sd[3 * SW_NNP + i];
    if constexpr (std::is_same<R, float>::value) {
        v.r = sf[0 * SW_NNP + i];
        v.b = sf[1 * SW_NNP + i];
        v.ux = sf[2 * SW_NNP + i];
        v.uy = sf[3 * SW_NNP + i];
        v.W = sf[4 * SW_NNP + i];
    } else {
        v.r = (R)v.rho;
        v.b = (R)v.beta;
        v.ux = (R)sd[4 * SW_NNP + i];
        v.uy = (R)sd[5 * SW_NNP + i];
        v.W = (R)sd[6 * SW_NNP + i];
    }
    return v;
}

template <typename R, int P, int WW>
__global__ void __launch_bounds__(256) k_sweep(ProbArg pa, Phys ph, const double *__restrict__ q,
                                               const float *__restrict__ q32, R *__restrict__ iflux, int dir,
                                               long long ntiles)
{
    using LY = SweepLayout<R, P>;
    using SH = SweepShape<P, WW>;
    constexpr bool F32 = LY::F32;
    using MT = typename std::conditional<F32, float, double>::type;
    constexpr int HL = SH::HL, HR = SH::HR, TA = SH::TA;
    extern __shared__ __align__(16) unsigned char sw_smem[];
    const int NW = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *sd = (double *)sw_smem + (size_t)w * LY::NF64 * SW_NNP;
    float *sf = (float *)((double *)sw_smem + (size_t)NW * LY::NF64 * SW_NNP) + (size_t)w * LY::NF32 * SW_NNP;
    R *spr = (R *)((float *)((double *)sw_smem + (size_t)NW * LY::NF64 * SW_NNP) + (size_t)NW * LY::NF32 * SW_NNP) +
             (size_t)w * LY::PAIR_VALUES;
    const MT *sMt = F32 ? (const MT *)(sf + 7 * SW_NNP) : (const MT *)(sd + 7 * SW_NNP);
    const MT *sMx = F32 ? (const MT *)(sf + 8 * SW_NNP) : (const MT *)(sd + 8 * SW_NNP);
    const MT *sMy = F32 ? (const MT *)(sf + 9 * SW_NNP) : (const MT *)(sd + 9 * SW_NNP);
    const R gm1inv = (R)(1.0 / (ph.gamma - 1.0));
    const R ig = (R)ph.gm1i, c1g = (R)ph.gamma * ig;   // as es_dissipation forms them

    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        ProbDesc D;
        long long lb;
        locate_tile(pa, t, D, lb);
        const Geom &g = D.g;
        const double *qq = q + (long long)NQ * D.op;
        const float *qq32 = F32 ? q32 + (long long)NQ32 * D.op : nullptr;
        R *fl = iflux + (long long)2 * 5 * D.op;
        const int nd = dir == 0 ? g.nx : g.ny, no = dir == 0 ? g.ny : g.nx;
        const long long S = (nd + 1 + TA - 1) / TA;
        const int seg = (int)(lb % S), grp = (int)(lb / S);
        const int L0 = -1 + seg * TA;
        const int Llast = min(L0 + TA - 1, nd - 1);    // last interface (left node) of the segment
        const int nlo = L0 - HL, nn = Llast + HR - nlo + 1;
        const int line = grp * NW + w;

        // stage the segment's nodes: [nlo, Llast + HR] along the sweep lies in
        // the padded range [-GH, nd - 1 + GH] since HL, HR <= GH
        if (dir == 0) {
            if (line < no)
                for (int e = lane; e < nn; e += 32)
                    sweep_stage<R>(g, qq, qq32, pidx(g, nlo + e, line), 0, c1g, ig, sd, sf, e);
        } else {
            for (int e = threadIdx.x; e < nn * NW; e += blockDim.x) {
                const int ww = e % NW, node = e / NW;
                if (grp * NW + ww < no)
                    sweep_stage<R>(g, qq, qq32, pidx(g, grp * NW + ww, nlo + node), 1, c1g, ig,
                                   (double *)sw_smem + (size_t)ww * LY::NF64 * SW_NNP,
                                   (float *)((double *)sw_smem + (size_t)NW * LY::NF64 * SW_NNP) +
                                       (size_t)ww * LY::NF32 * SW_NNP,
                                   node);
            }
        }
        __syncthreads();

        if (line < no) {
            // the anchors' pair fluxes (k_pairs): lane -> anchor L0 - (p - 1) + lane
            const int A = L0 - (P - 1) + lane;
            if (A <= Llast) {
                const int ia = A - nlo;
                NodeV<R> l = sweep_node<R>(sd, sf, ia);
                const MT mtl = sMt[ia], mxl = sMx[ia], myl = sMy[ia];
#pragma unroll
                for (int n = 1; n <= P; ++n) {
                    const int ir = ia + n;
                    NodeV<R> r = sweep_node<R>(sd, sf, ir);
                    R mt = (R)((MT)0.5 * (mtl + sMt[ir]));
                    R mx = (R)((MT)0.5 * (mxl + sMx[ir]));
                    R my = (R)((MT)0.5 * (myl + sMy[ir]));
                    R out[4];
                    ec_pair<R>(l, r, mt, mx, my, gm1inv, ph.ln_thr, out);
#pragma unroll
                    for (int a = 0; a < 4; ++a) spr[((n - 1) * 4 + a) * 32 + lane] = out[a];
                }
            }
            __syncwarp();

            // the interfaces (k_iface): lane -> interface between L = L0 + lane and L + 1
            const int L = L0 + lane;
            if (lane < TA && L <= Llast) {
                const int i0 = L - nlo;
                R F[4] = {(R)0, (R)0, (R)0, (R)0};
                MT Ft = (MT)0;
#pragma unroll
                for (int n = 1; n <= P; ++n) {
                    R Fs[4] = {(R)0, (R)0, (R)0, (R)0};
                    MT Fts = (MT)0;
#pragma unroll
                    for (int s = 0; s < n; ++s) {
                        const R *pr = spr + (n - 1) * 4 * 32 + (lane + P - 1 - s);
#pragma unroll
                        for (int a = 0; a < 4; ++a) Fs[a] += pr[a * 32];
                        Fts += (MT)0.5 * (sMt[i0 - s] + sMt[i0 - s + n]);
                    }
                    const R an = (R)ph.alpha[n - 1];
#pragma unroll
                    for (int a = 0; a < 4; ++a) F[a] += an * Fs[a];
                    Ft += (MT)ph.alpha[n - 1] * Fts;
                }
                if constexpr (WW > 0) {
                    const int i1 = i0 + 1;
                    const R nvx = (R)((MT)0.5 * (sMx[i0] + sMx[i1])), nvy = (R)((MT)0.5 * (sMy[i0] + sMy[i1]));
                    const R jt = (R)((MT)0.5 * (sMt[i0] + sMt[i1]));
                    const double rho0 = sd[0 * SW_NNP + i0], rho1 = sd[0 * SW_NNP + i1];
                    const double lnr0 = sd[2 * SW_NNP + i0], lnr1 = sd[2 * SW_NNP + i1];
                    R diss[4];
                    if constexpr (F32) {
                        SmemStencil<float> st{sf, i0 - (WW - 1) / 2};
                        es_dissipation<R, double, WW>(nvx, nvy, jt, rho0, rho1, lnr0, lnr1, sf[0 * SW_NNP + i0],
                                                      sf[0 * SW_NNP + i1], st, ph, diss);
                    } else {
                        SmemStencil<double> st{sd, i0 - (WW - 1) / 2};
                        es_dissipation<R, double, WW>(nvx, nvy, jt, rho0, rho1, lnr0, lnr1, (R)rho0, (R)rho1, st, ph,
                                                      diss);
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a) F[a] -= diss[a];
                }
                const long long c0 = dir == 0 ? pidx(g, L, line) : pidx(g, line, L);
                R *out = fl + (long long)(dir * 5) * g.P + c0;
#pragma unroll
                for (int a = 0; a < 4; ++a) out[a * g.P] = F[a];
                out[4 * g.P] = (R)Ft;
            }
        }
        __syncthreads();   // the next tile restages the arrays
    }
}

template <typename R, int P, int WW>
static void launch_sweep_pw(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, R *iflux, int dir,
                            cudaStream_t st)
{
    const size_t smem = (size_t)(L.bs / 32) * SweepLayout<R, P>::bytes_per_warp;
    if (smem > 48 * 1024) {   // once per device and instantiation: allow more than 48 KB
        static bool attr[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev < 0 || dev >= 64 || !attr[dev]) {
            cudaFuncSetAttribute(k_sweep<R, P, WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (dev >= 0 && dev < 64) attr[dev] = true;
        }
    }
    k_sweep<R, P, WW><<<L.nblk, L.bs, smem, st>>>(L.pa, ph, q, q32, iflux, dir, tiles_of(L));
}

template <typename R, int P>
static void launch_sweep_p(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, R *fl, int dir,
                           cudaStream_t st)
{
    switch (ph.w) {
    case 0: launch_sweep_pw<R, P, 0>(L, ph, q, q32, fl, dir, st); break;
    case 3: launch_sweep_pw<R, P, 3>(L, ph, q, q32, fl, dir, st); break;
    default: launch_sweep_pw<R, P, 5>(L, ph, q, q32, fl, dir, st); break;
    }
}

template <typename R>
void launch_sweep_t(const LaunchDom &L, const Phys &ph, const double *q, const float *q32, void *iflux, int dir,
                    cudaStream_t st)
{
    R *fl = (R *)iflux;
    switch (ph.p) {
    case 1: launch_sweep_p<R, 1>(L, ph, q, q32, fl, dir, st); break;
    case 2: launch_sweep_p<R, 2>(L, ph, q, q32, fl, dir, st); break;
    default: launch_sweep_p<R, 3>(L, ph, q, q32, fl, dir, st); break;
    }
}

template <typename R, int P, int WW>
static int sweep_occ(int bs)
{
    int n = 0;
    const size_t smem = (size_t)(bs / 32) * SweepLayout<R, P>::bytes_per_warp;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_sweep<R, P, WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<R, P, WW>, bs, smem) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

template <typename R, int P>
static int sweep_occ_p(int w, int bs)
{
    return w == 0 ? sweep_occ<R, P, 0>(bs) : (w == 3 ? sweep_occ<R, P, 3>(bs) : sweep_occ<R, P, 5>(bs));
}

// resident blocks per SM of the sweep kernel at block size bs
template <typename R>
int sweep_occupancy_t(int p, int w, int bs)
{
    return p == 1 ? sweep_occ_p<R, 1>(w, bs) : (p == 2 ? sweep_occ_p<R, 2>(w, bs) : sweep_occ_p<R, 3>(w, bs));
}

}  // namespace esmm
