// esmm_mhd.cuh -- device arithmetic and kernels of the RMHD scheme (Duan &
// Tang, arXiv 2107.12027): primitive recovery, the two-point EC flux with its
// Godunov-Powell term, the scaled eigenvectors of the symmetrized system, the
// ES interface flux, the Powell source in the update, and the CFL radius.
//
// State: cons [8][N] = J (D, m_1, m_2, m_3, E, B_1, B_2, B_3), primitives
// (rho, v_1, v_2, v_3, p, B_1, B_2, B_3).  Node data extend the RHD layout of
// esmm_device.cuh (indices 0..13 keep their meaning) by u_3 and B_1..B_3, so
// the mesh, temporal-metric and totals kernels serve both systems.
// Device arithmetic and the templated kernels; the 2D instantiations live in
// esmm_mhd.cu and the 3D kernels (esmm_3d.cu) reuse the arithmetic.
#pragma once

#include <type_traits>

#include "esmm_device.cuh"
#include "esmm_launch.h"

namespace esmm {

enum { QM_UZ = NQ, QM_B1, QM_B2, QM_B3, NQM };   // 18 node arrays (NQ_MHD)
constexpr int NFM = 10;                          // interface values per direction: F[8], J xi_t, B~ (NF_MHD)

// ---------------------------------------------------------------------------
// Primitive recovery (FP64).  Newton on Z = rho h W^2 with bisection on
// [0, Gamma E]; with S = m.B,
//   v.B = S/Z,  |v|^2 = (|m|^2 + (2Z + |B|^2) S^2/Z^2)/(Z + |B|^2)^2,
//   p = (Gamma-1)/Gamma (Z/W^2 - D/W),
//   f(Z) = Z - p + |B|^2 (1 + |v|^2)/2 - S^2/(2 Z^2) - E,
// a trial Z with |v|^2 >= 1 lying below the root.  Stops when a step moves Z
// by at most 1e-15 (E + Z), or where |f| <= 2e-15 (E + Z), f's rounding
// level (a root, whose tiny steps the open bracket would otherwise reject).
// Z0: warm start (ignored outside the bracket).  Quotients are taken through
// reciprocals, and the Newton step divides by df through an FP32 reciprocal
// (the slope only steers the step; f, which decides the stopping, is FP64).
// Returns 0, 1 (non-admissible) or 2 (iteration cap).
__device__ __forceinline__ int cons2prim_mhd(double gam, const double U[8], double Z0, double w[8], double &Zout)
{
    const double D = U[0], E = U[4];
    const double m0 = U[1], m1 = U[2], m2_ = U[3], B0 = U[5], B1 = U[6], B2_ = U[7];
    const double m2 = m0 * m0 + m1 * m1 + m2_ * m2_;
    const double B2 = B0 * B0 + B1 * B1 + B2_ * B2_;
    const double S = m0 * B0 + m1 * B1 + m2_ * B2_;
    const double S2 = S * S;
    const double g = (gam - 1.0) / gam;
    for (int a = 0; a < 8; ++a) w[a] = 0.0;
    Zout = 0.0;
    if (!(D > 0.0) || !(E > 0.0)) return 1;
    double lo = 0.0, hi = gam * E;
    double Z = (Z0 > lo && Z0 < hi) ? Z0 : 0.5 * (lo + hi);
    int ok = 0;
    for (int it = 0; it < 300; ++it) {
        double ZB = Z + B2;
        double iZ = __drcp_rn(Z);
        double N = m2 + (2.0 * Z + B2) * S2 * iZ * iZ;
        double iZB = __drcp_rn(ZB);
        double v2 = N * iZB * iZB;
        double Zn;
        if (!(v2 < 1.0)) {
            lo = Z;
            Zn = 0.5 * (lo + hi);
        } else {
            double iW2 = 1.0 - v2, rs = rsqrt(iW2), iW = iW2 * rs;
            double p = g * (Z * iW2 - D * iW);
            double f = Z - p + 0.5 * B2 * (1.0 + v2) - 0.5 * S2 * iZ * iZ - E;
            double dN = -2.0 * S2 * iZ * iZ - 2.0 * B2 * S2 * iZ * iZ * iZ;
            double dv2 = dN * iZB * iZB - 2.0 * N * iZB * iZB * iZB;
            double dp = g * (iW2 - Z * dv2 + 0.5 * D * dv2 * rs);
            double df = 1.0 - dp + 0.5 * B2 * dv2 + S2 * iZ * iZ * iZ;
            if (fabs(f) <= 2.0e-15 * (E + Z)) { ok = 1; break; }   // residual at rounding level
            Zn = Z;                          // f = 0: Z is a root
            if (f != 0.0) {
                if (f < 0.0) lo = Z; else hi = Z;
                Zn = Z - f * f2d_int(__frcp_rn(d2f_int(df)));
                if (!(Zn > lo && Zn < hi)) Zn = 0.5 * (lo + hi);
            }
        }
        if (fabs(Zn - Z) <= 1.0e-15 * (E + Zn)) { Z = Zn; ok = 1; break; }
        Z = Zn;
    }
    double ZB = Z + B2, iZ = __drcp_rn(Z), iZB = __drcp_rn(ZB);
    double v2 = (m2 + (2.0 * Z + B2) * S2 * iZ * iZ) * iZB * iZB;
    if (!(v2 < 1.0)) return 1;
    double iW2 = 1.0 - v2, iW = sqrt(iW2);
    double vB = S * iZ;
    w[0] = D * iW;
    w[1] = (m0 + vB * B0) * iZB;
    w[2] = (m1 + vB * B1) * iZB;
    w[3] = (m2_ + vB * B2_) * iZB;
    w[4] = g * (Z * iW2 - D * iW);
    w[5] = B0; w[6] = B1; w[7] = B2_;
    Zout = Z;
    if (!(w[4] > 0.0)) return 1;
    return ok ? 0 : 2;
}

// U(w), F_1(w) and V(w) (eq. RMHDdiv2, Sec. 2), generic in the number type
// so that dual numbers give directional derivatives.
template <typename T> __device__ __forceinline__ T lg(T x);
template <> __device__ __forceinline__ double lg<double>(double x) { return log(x); }
template <> __device__ __forceinline__ dual lg<dual>(dual x) { return dual(log(x.v), x.d * __drcp_rn(x.v)); }
template <> __device__ __forceinline__ fdual lg<fdual>(fdual x) { return fdual(logf(x.v), x.d * __frcp_rn(x.v)); }
template <> __device__ __forceinline__ hdual lg<hdual>(hdual x)
{
    double r = __drcp_rn(x.v);
    return hchain(x, log(x.v), r, -r * r);
}

template <typename T>
__device__ __forceinline__ void mhd_UFV(double gam, const T w[8], T U[8], T F[8], T V[8])
{
    T rho = w[0], p = w[4];
    T v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
    T iW2 = 1.0 - v2;
    T W = rsq<T>(iW2);                 // (reciprocals and rsqrt: no FP64 quotient)
    T W2 = W * W;
    T vB = w[1] * w[5] + w[2] * w[6] + w[3] * w[7];
    T B2 = w[5] * w[5] + w[6] * w[6] + w[7] * w[7];
    T bb = B2 * iW2 + vB * vB;
    T rhoh = rho + (gam / (gam - 1.0)) * p;
    T pt = p + 0.5 * bb;
    T Q = rhoh * W2 + B2;
    U[0] = rho * W;
#pragma unroll
    for (int k = 0; k < 3; ++k) U[1 + k] = Q * w[1 + k] - vB * w[5 + k];
    U[4] = rhoh * W2 - pt + B2;
#pragma unroll
    for (int k = 0; k < 3; ++k) U[5 + k] = w[5 + k];
    F[0] = U[0] * w[1];
#pragma unroll
    for (int k = 0; k < 3; ++k) F[1 + k] = U[1 + k] * w[1] - w[5] * (w[5 + k] * iW2 + vB * w[1 + k]);
    F[1] = F[1] + pt;
    F[4] = U[1];
#pragma unroll
    for (int k = 0; k < 3; ++k) F[5 + k] = w[1] * w[5 + k] - w[5] * w[1 + k];
    T beta = rho * rcp<T>(p);
    T s = lg<T>(p) - gam * lg<T>(rho);
    V[0] = (gam - s) * (1.0 / (gam - 1.0)) + beta;
#pragma unroll
    for (int k = 0; k < 3; ++k) V[1 + k] = beta * W * w[1 + k];
    V[4] = -beta * W;
    const T bW = beta * iW2 * W;       // beta / W
#pragma unroll
    for (int k = 0; k < 3; ++k) V[5 + k] = bW * (w[5 + k] + W2 * w[1 + k] * vB);
}

// Images (dU, dV, dF~) of the primitive perturbation dir at w, with the
// Godunov-Powell column: dF~ = dF_1 + Phi'(V) dB_1, in the working precision R.
template <typename R>
__device__ __forceinline__ void mhd_images(double gam, const R w[8], const R dir[8], const R Pp[8], R dU[8], R dV[8],
                                           R dF[8])
{
    using D = typename DualOf<R>::type;
    D wd[8], U[8], F[8], V[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) wd[a] = img_seed(w[a], dir[a]);
    mhd_UFV<D>(gam, wd, U, F, V);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        dU[a] = img_part(U[a]);
        dV[a] = img_part(V[a]);
        dF[a] = img_part(F[a]) + Pp[a] * dir[5];
    }
}

template <typename R>
__device__ __forceinline__ R dot8(const R *a, const R *b)
{
    R s = (R)0;
#pragma unroll
    for (int r = 0; r < 8; ++r) s += a[r] * b[r];
    return s;
}

// f(0) ... f(n - 1), in a rolled loop in the FP32 instances, whose kernels are
// limited by instruction fetch (the unrolled copies of these loop bodies do
// not fit the instruction cache); as the compiler chooses otherwise.
template <typename R, typename F>
__device__ __forceinline__ void each_index(int n, F &&f)
{
    if constexpr (std::is_same<R, float>::value) {
#pragma unroll 1
        for (int i = 0; i < n; ++i) f(i);
    } else {
        for (int i = 0; i < n; ++i) f(i);
    }
}

// Phi'(V) = (0, B/W^2 + v (v.B), v.B, v) (eq. Phi)
template <typename R>
__device__ __forceinline__ void mhd_phiprime(const R w[8], R P[8])
{
    R iW2 = (R)1 - (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
    R vB = w[1] * w[5] + w[2] * w[6] + w[3] * w[7];
    P[0] = (R)0;
#pragma unroll
    for (int k = 0; k < 3; ++k) P[1 + k] = w[5 + k] * iW2 + w[1 + k] * vB;
    P[4] = vB;
#pragma unroll
    for (int k = 0; k < 3; ++k) P[5 + k] = w[1 + k];
}

// Scaled eigenvectors of the symmetrized x_1 system (Sec. 4) at the rotated
// primitive state w: lam[8] and R[8][8] (row = component, column = wave)
// with R R^T = dU/dV.  Construction (as the paper only cites formulas):
// <a, b> = dU(a).dV(b), k(a, b) = dV(a).dF~(b); the entropy wave e_rho and
// the divergence wave dB = e_1 - v_1 v have speed v_1; the other six waves
// span the <.,.> complement of y_a = e_a - projections (a = v_1, v_2, v_3,
// p, B_2, B_3) and come from cyclic Jacobi on C = L^-1 K L^-T (G = L L^T);
// clusters of speeds closer than CLUSTER_TOL get the canonical basis of
// their span (Gram-Schmidt, in index order, of the projected C-space unit
// vectors whose remaining squared norm is at least 1/8: continuous in the
// span, unlike a largest-norm choice, which switches on the exact ties of
// symmetric states).
constexpr double MHD_CLUSTER_TOL = 1.0e-5;

// Cyclic Jacobi on the symmetric 6 x 6 C (in place: its diagonal becomes the
// eigenvalues), accumulating the rotations in Q when want_vectors.
template <typename S>
__device__ __forceinline__ void jacobi6(S C[6][6], S Q[6][6], bool want_vectors)
{
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) Q[a][b] = a == b ? (S)1 : (S)0;
    // converged when the off-diagonal part is at rounding level: (1e-15)^2
    // of the diagonal in FP64, (1e-6)^2 in FP32 (the next sweep squares it)
    const S conv = sizeof(S) == 4 ? (S)1.0e-12 : (S)1.0e-30;
    for (int sweep = 0; sweep < 50; ++sweep) {
        S off = (S)0, dg = (S)0;
        for (int a = 0; a < 6; ++a) {
            dg += C[a][a] * C[a][a];
            for (int b = a + 1; b < 6; ++b) off += C[a][b] * C[a][b];
        }
        if (off <= conv * dg) break;
        // The rotation loops stay rolled: fully unrolled, this sweep came out
        // of nvcc 13.0 -O3 (sm_103a) as a non-similarity transform (wrong
        // eigenvalues; the host build and the -G build of the same source are
        // right), so unrolling is disabled here.
#pragma unroll 1
        for (int p = 0; p < 5; ++p)
#pragma unroll 1
            for (int q = p + 1; q < 6; ++q) {
                if (C[p][q] == (S)0) continue;
                // (reciprocals for the rotation's quotients: FP64 divisions
                // cost ~15 FP64-pipe instructions each on this GPU).  A tiny
                // C_pq can have an infinite reciprocal: equal diagonals then
                // take theta = 0 (as the quotient 0 / (2 C_pq) does), unequal
                // ones theta = +-inf, hence t = 0 (no rotation)
                const S diff = C[q][q] - C[p][p];
                S theta = diff == (S)0 ? (S)0 : diff * ((S)0.5 * rcp<S>(C[p][q]));
                S t = (theta >= (S)0 ? (S)1 : (S)-1) * rcp<S>(fab<S>(theta) + sq_rt<S>(theta * theta + (S)1));
                S cs = rsq<S>(t * t + (S)1), sn = t * cs;
#pragma unroll 1
                for (int k = 0; k < 6; ++k) {
                    S ckp = C[k][p], ckq = C[k][q];
                    C[k][p] = cs * ckp - sn * ckq;
                    C[k][q] = sn * ckp + cs * ckq;
                }
#pragma unroll 1
                for (int k = 0; k < 6; ++k) {
                    S cpk = C[p][k], cqk = C[q][k];
                    C[p][k] = cs * cpk - sn * cqk;
                    C[q][k] = sn * cpk + cs * cqk;
                }
                if (want_vectors)
#pragma unroll 1
                    for (int k = 0; k < 6; ++k) {
                        S qkp = Q[k][p], qkq = Q[k][q];
                        Q[k][p] = cs * qkp - sn * qkq;
                        Q[k][q] = sn * qkp + cs * qkq;
                    }
            }
    }
}

template <typename R>
static __device__ __noinline__ void eigen_mhd(double gam, const R w[8], R lam[8], R Rv[8][8], bool want_vectors)
{
    R Pp[8];
    mhd_phiprime(w, Pp);
    const R v1 = w[1];
    R a_rho[8] = {(R)1, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0};
    R a_div[8] = {(R)0, (R)0, (R)0, (R)0, (R)0, (R)1 - v1 * v1, -v1 * w[2], -v1 * w[3]};
    R Ur[8], Vr[8], Fr[8], Ud[8], Vd[8], Fd[8];
    mhd_images(gam, w, a_rho, Pp, Ur, Vr, Fr);
    mhd_images(gam, w, a_div, Pp, Ud, Vd, Fd);
    const R n_rho = dot8(Ur, Vr), n_div = dot8(Ud, Vd);
    const R in_rho = rcp<R>(n_rho), in_div = rcp<R>(n_div);
    const int comp[6] = {1, 2, 3, 4, 6, 7};
    R Uy[6][8], Vy[6][8], Fy[6][8];
    each_index<R>(6, [&](int a) {
        R e[8] = {(R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0};
        e[comp[a]] = (R)1;
        R Ue[8], Ve[8], Fe[8];
        mhd_images(gam, w, e, Pp, Ue, Ve, Fe);
        R cr = dot8(Ue, Vr) * in_rho, cd = dot8(Ue, Vd) * in_div;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            Uy[a][r] = Ue[r] - cr * Ur[r] - cd * Ud[r];
            Vy[a][r] = Ve[r] - cr * Vr[r] - cd * Vd[r];
            Fy[a][r] = Fe[r] - cr * Fr[r] - cd * Fd[r];
        }
        if constexpr (std::is_same<R, float>::value) {
            // FP32: scale y_a to unit <y_a, y_a> (the Gram diagonal spans
            // many decades at large W); C = L^-1 K L^-T is unchanged by it
            R sa = rsq<R>(dot8(Uy[a], Vy[a]));
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                Uy[a][r] *= sa;
                Vy[a][r] *= sa;
                Fy[a][r] *= sa;
            }
        }
    });
    R Gm[6][6], C[6][6];
    each_index<R>(6, [&](int a) {
        each_index<R>(a + 1, [&](int b) {
            R g = (R)0.5 * (dot8(Uy[a], Vy[b]) + dot8(Uy[b], Vy[a]));
            R k = (R)0.5 * (dot8(Vy[a], Fy[b]) + dot8(Vy[b], Fy[a]));
            Gm[a][b] = Gm[b][a] = g;
            C[a][b] = C[b][a] = k;
        });
    });
    // Cholesky G = L L^T (lower triangle of Gm), with the reciprocals of
    // its diagonal (idg) serving every division of the factor and the solves
    R idg[6];
    for (int j = 0; j < 6; ++j) {
        R d = Gm[j][j];
        for (int k = 0; k < j; ++k) d -= Gm[j][k] * Gm[j][k];
        if constexpr (std::is_same<R, float>::value)
            if (!(d > (R)1.0e-12)) d = (R)1.0e-12;   // FP32: keep the factor finite
        Gm[j][j] = sq_rt<R>(d);
        idg[j] = rcp<R>(Gm[j][j]);
        for (int i = j + 1; i < 6; ++i) {
            R s = Gm[i][j];
            for (int k = 0; k < j; ++k) s -= Gm[i][k] * Gm[j][k];
            Gm[i][j] = s * idg[j];
        }
    }
    // C <- L^-1 K L^-T (column solves, then row solves)
    for (int c = 0; c < 6; ++c)
        for (int i = 0; i < 6; ++i) {
            R s = C[i][c];
            for (int k = 0; k < i; ++k) s -= Gm[i][k] * C[k][c];
            C[i][c] = s * idg[i];
        }
    for (int r = 0; r < 6; ++r)
        for (int i = 0; i < 6; ++i) {
            R s = C[r][i];
            for (int k = 0; k < i; ++k) s -= Gm[i][k] * C[r][k];
            C[r][i] = s * idg[i];
        }
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < a; ++b) C[a][b] = C[b][a] = (R)0.5 * (C[a][b] + C[b][a]);
    int ord[6] = {0, 1, 2, 3, 4, 5};
    R E6[6][6];
    if constexpr (std::is_same<R, dual>::value) {
        // Adjoint tangent: Jacobi on the values; first-order perturbation
        // theory for the tangent.  With M = Q^T C' Q (C' = C.d), an eigenvalue
        // moves by M_ii and eigenvector i by sum_j M_ji / (lam_i - lam_j) e_j
        // over the j outside i's cluster: inside a cluster only the span is
        // defined, and the canonical basis below is a function of the span.
        double Cv[6][6], Qv[6][6], M[6][6];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) Cv[i][j] = C[i][j].v;
        jacobi6<double>(Cv, Qv, true);
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 6; ++k)
                    for (int l = 0; l < 6; ++l) acc += Qv[k][i] * C[k][l].d * Qv[l][j];
                M[i][j] = acc;
            }
        for (int a = 0; a < 6; ++a)
            for (int b = a + 1; b < 6; ++b)
                if (Cv[ord[b]][ord[b]] < Cv[ord[a]][ord[a]]) { int t = ord[a]; ord[a] = ord[b]; ord[b] = t; }
        int cl[6];   // cluster id of each sorted wave
        cl[0] = 0;
        for (int m = 1; m < 6; ++m)
            cl[m] = cl[m - 1] + (Cv[ord[m]][ord[m]] - Cv[ord[m - 1]][ord[m - 1]] < MHD_CLUSTER_TOL ? 0 : 1);
        for (int m = 0; m < 6; ++m) {
            const int i = ord[m];
            const double li = Cv[i][i];
            lam[2 + m] = dual(li, M[i][i]);
            if (!want_vectors) continue;
            for (int r = 0; r < 6; ++r) {
                double t = 0.0;
                for (int n = 0; n < 6; ++n) {
                    if (cl[n] == cl[m]) continue;
                    const int j = ord[n];
                    t += M[j][i] / (li - Cv[j][j]) * Qv[r][j];
                }
                E6[r][m] = dual(Qv[r][i], t);
            }
        }
        lam[0] = v1;
        lam[1] = v1;
        if (!want_vectors) return;
    } else {
        R Q[6][6];
        jacobi6<R>(C, Q, want_vectors);
        for (int a = 0; a < 6; ++a)
            for (int b = a + 1; b < 6; ++b)
                if (C[ord[b]][ord[b]] < C[ord[a]][ord[a]]) { int t = ord[a]; ord[a] = ord[b]; ord[b] = t; }
        lam[0] = v1;
        lam[1] = v1;
        for (int m = 0; m < 6; ++m) lam[2 + m] = C[ord[m]][ord[m]];
        if (!want_vectors) return;
        for (int m = 0; m < 6; ++m)
            for (int r = 0; r < 6; ++r) E6[r][m] = Q[r][ord[m]];
    }
    int start = 0;
    while (start < 6) {
        int end = start + 1;
        while (end < 6 && val(lam[2 + end]) - val(lam[1 + end]) < MHD_CLUSTER_TOL) ++end;
        const int k = end - start;
        if (k > 1) {
            // Gram-Schmidt in index order of the C-space unit vectors projected
            // on the cluster's span, taking those with remaining squared norm
            // >= 1/8 (k of them always are: the six squared norms sum to k)
            R z[6][6], basis[6][6];
            for (int i = 0; i < 6; ++i)
                for (int c = 0; c < k; ++c) z[i][c] = E6[i][start + c];
            int nt = 0;
            for (int i = 0; i < 6 && nt < k; ++i) {
                R n2 = (R)0;
                for (int c = 0; c < k; ++c) n2 += z[i][c] * z[i][c];
                if (!(val(n2) >= 0.125)) continue;
                R inr = (R)1 / sq_rt<R>(n2);
                for (int c = 0; c < k; ++c) basis[nt][c] = z[i][c] * inr;
                for (int ii = i + 1; ii < 6; ++ii) {
                    R pr = (R)0;
                    for (int c = 0; c < k; ++c) pr += z[ii][c] * basis[nt][c];
                    for (int c = 0; c < k; ++c) z[ii][c] -= pr * basis[nt][c];
                }
                ++nt;
            }
            if (nt < k) {   // only for non-finite input: keep the Jacobi basis
                start = end;
                continue;
            }
            R nE[6][6];
            for (int t = 0; t < k; ++t)
                for (int r = 0; r < 6; ++r) {
                    R acc = (R)0;
                    for (int c = 0; c < k; ++c) acc += E6[r][start + c] * basis[t][c];
                    nE[r][t] = acc;
                }
            for (int t = 0; t < k; ++t)
                for (int r = 0; r < 6; ++r) E6[r][start + t] = nE[r][t];
        }
        start = end;
    }
    const R srho = rsq<R>(n_rho), sdiv = rsq<R>(n_div);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        Rv[r][0] = Ur[r] * srho;
        Rv[r][1] = Ud[r] * sdiv;
    }
    each_index<R>(6, [&](int m) {
        R s[6];
        for (int i = 5; i >= 0; --i) {
            R acc = E6[i][m];
            for (int k = i + 1; k < 6; ++k) acc -= Gm[k][i] * s[k];
            s[i] = acc * idg[i];
        }
        for (int r = 0; r < 8; ++r) {
            R acc = (R)0;
            for (int a = 0; a < 6; ++a) acc += s[a] * Uy[a][r];
            Rv[r][2 + m] = acc;
        }
    });
}

// ---------------------------------------------------------------------------
// Node values of one two-point flux argument: the log-mean arguments in FP64,
// the rest (with copies r, b of rho, beta) in the working precision R.
template <typename R>
struct NodeMT {
    typename LogT<R>::type rho, beta, lnr, lnb;   // FP64 (dual in the adjoint)
    R r, b, W, u[3], B[3];
};
using NodeM = NodeMT<double>;

template <typename R = double>
__device__ __forceinline__ NodeMT<R> load_node_m(const double *__restrict__ q, long long P, long long c)
{
    NodeMT<R> v;
    v.rho = q[Q_RHO * P + c];
    v.beta = q[Q_BETA * P + c];
    v.lnr = q[Q_LNR * P + c];
    v.lnb = q[Q_LNB * P + c];
    v.r = (R)v.rho;
    v.b = (R)v.beta;
    v.W = (R)q[Q_W * P + c];
    v.u[0] = (R)q[Q_UX * P + c];
    v.u[1] = (R)q[Q_UY * P + c];
    v.u[2] = (R)q[QM_UZ * P + c];
    v.B[0] = (R)q[QM_B1 * P + c];
    v.B[1] = (R)q[QM_B2 * P + c];
    v.B[2] = (R)q[QM_B3 * P + c];
    return v;
}

// Curvilinear two-point EC flux (Sec. 3.1) of one node pair:
//   out = mt U~ + sum_{j<NJ} m_j F~_j with the averaged metrics mt, m.
// U~: the paper's U~^RMHD with R_1 summed over three components and its
// magnetic term 1/2 {{W (b^k)^2}}; F~_j: coefficient matching with exact
// product-rule expansions, including the -{{B_j}}[[Phi]] term.  Here
// b = (B + (u.B) u)/W, b^0 = u.B, c = W b^0, v = u/W.
template <int NJ, typename R>
__device__ __forceinline__ void ec_pair_mhd(const NodeMT<R> &L, const NodeMT<R> &Rn, R gm1inv, double thr, R mt,
                                            const R m[3], R out[8])
{
    R rln, irln, bln, ibln;
    lmean<R, typename LogT<R>::type>(L.rho, Rn.rho, L.lnr, Rn.lnr, L.r, Rn.r, thr, rln, irln);
    lmean<R, typename LogT<R>::type>(L.beta, Rn.beta, L.lnb, Rn.lnb, L.b, Rn.b, thr, bln, ibln);
    const R half = (R)0.5;
    R bL[3], bR[3], vL[3], vR[3];
    // b^0 = W (v.B) = u.B
    R b0L = L.u[0] * L.B[0] + L.u[1] * L.B[1] + L.u[2] * L.B[2];
    R b0R = Rn.u[0] * Rn.B[0] + Rn.u[1] * Rn.B[1] + Rn.u[2] * Rn.B[2];
    R iWL = rcp<R>(L.W), iWR = rcp<R>(Rn.W);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        bL[k] = (L.B[k] + b0L * L.u[k]) * iWL;
        bR[k] = (Rn.B[k] + b0R * Rn.u[k]) * iWR;
        vL[k] = L.u[k] * iWL;
        vR[k] = Rn.u[k] * iWR;
    }
    const R rho_m = half * (L.r + Rn.r), beta_m = half * (L.b + Rn.b), W_m = half * (L.W + Rn.W);
    R u_m[3], b_m[3], bsq_m[3], Wbsq_m[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u_m[k] = half * (L.u[k] + Rn.u[k]);
        b_m[k] = half * (bL[k] + bR[k]);
        bsq_m[k] = half * (bL[k] * bL[k] + bR[k] * bR[k]);
        Wbsq_m[k] = half * (L.W * bL[k] * bL[k] + Rn.W * bR[k] * bR[k]);
    }
    const R c_m = half * (L.W * b0L + Rn.W * b0R);
    const R Wb0sq_m = half * (L.W * b0L * b0L + Rn.W * b0R * b0R);
    const R b0_m = half * (b0L + b0R);
    const R usq = u_m[0] * u_m[0] + u_m[1] * u_m[1] + u_m[2] * u_m[2];
    const R Lam = W_m * W_m - usq;
    const R alpha0 = (R)1 + gm1inv * ibln;
    const R iW_m = rcp<R>(W_m), ibeta_m = rcp<R>(beta_m), iLam = rcp<R>(Lam);
    const R bsq_sum = bsq_m[0] + bsq_m[1] + bsq_m[2];
    // U~
    R Ut[8];
    {
        const R alpha1 = rho_m + half * beta_m * bsq_sum + half * beta_m * Wb0sq_m * iW_m;
        const R U1 = rln * W_m;
        R UB[3], Rk[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) UB[k] = (W_m * W_m * b_m[k] - c_m * u_m[k]) * iW_m;
        R R1 = -alpha0 * U1 - half * Wb0sq_m;
#pragma unroll
        for (int k = 0; k < 3; ++k) R1 += half * Wbsq_m[k] - b_m[k] * UB[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) Rk[k] = (alpha1 * u_m[k] - beta_m * c_m * b_m[k]) * iW_m;
        const R U5 = (u_m[0] * Rk[0] + u_m[1] * Rk[1] + u_m[2] * Rk[2] - beta_m * R1) * W_m * ibeta_m * iLam;
        Ut[0] = U1;
#pragma unroll
        for (int k = 0; k < 3; ++k) Ut[1 + k] = u_m[k] * U5 * iW_m + Rk[k] * ibeta_m;
        Ut[4] = U5;
#pragma unroll
        for (int k = 0; k < 3; ++k) Ut[5 + k] = UB[k];
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) out[a] = mt * Ut[a];
    // F~_j, j = 1..NJ
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const R mj = m[j];
        R ujbsq = (R)0;
#pragma unroll
        for (int k = 0; k < 3; ++k) ujbsq += half * (L.u[j] * bL[k] * bL[k] + Rn.u[j] * bR[k] * bR[k]);
        const R ujb0sq = half * (L.u[j] * b0L * b0L + Rn.u[j] * b0R * b0R);
        const R vj_m = half * (vL[j] + vR[j]);
        const R Bj_m = half * (L.B[j] + Rn.B[j]);
        R r_beta = (R)0, r_u[3] = {(R)0, (R)0, (R)0}, r_b[3];
        R cW = (R)0, cc = (R)0;
        r_u[j] += rho_m;
        r_beta += half * ujbsq;
        r_u[j] += half * beta_m * bsq_sum;
#pragma unroll
        for (int k = 0; k < 3; ++k) r_b[k] = beta_m * u_m[j] * b_m[k];
        r_beta -= half * ujb0sq;
        cc -= beta_m * vj_m * c_m * iW_m;
        cW += beta_m * vj_m * Wb0sq_m * iW_m;        // both [[W]] terms of -(1/2)[[beta u_j (b^0)^2]]
        r_u[j] -= half * beta_m * Wb0sq_m * iW_m;
        r_beta -= Bj_m * b0_m;
        cc -= Bj_m * beta_m * iW_m;
        cW += Bj_m * beta_m * b0_m * iW_m;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            r_u[k] += cW * u_m[k] * iW_m + cc * b_m[k];
            r_b[k] += cc * u_m[k];
        }
        R F[8];
        F[0] = rln * u_m[j];
#pragma unroll
        for (int k = 0; k < 3; ++k) F[5 + k] = r_b[k] * ibeta_m;
        R acc = alpha0 * F[0] - r_beta;
#pragma unroll
        for (int k = 0; k < 3; ++k) acc += u_m[k] * r_u[k] * ibeta_m + b_m[k] * F[5 + k];
        F[4] = W_m * acc * iLam;
#pragma unroll
        for (int k = 0; k < 3; ++k) F[1 + k] = r_u[k] * ibeta_m + u_m[k] * F[4] * iW_m;
#pragma unroll
        for (int a = 0; a < 8; ++a) out[a] += mj * F[a];
    }
}

// ---------------------------------------------------------------------------
// Per padded node: recovery (warm-started from zg_in), node values, metrics.
template <int P>
__global__ void k_node_mhd(ProbArg pa, double gam, const double *__restrict__ cons, const double *__restrict__ J,
                           const double *__restrict__ x, const double *__restrict__ xdot,
                           const double *__restrict__ zg_in, double *__restrict__ zg_out, double *__restrict__ q,
                           int *__restrict__ status, const double *__restrict__ inflow, int f32_logs)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long t = lb * blockDim.x + threadIdx.x;
    if (t >= g.P) return;
    int I = (int)(t % g.px) - GH, Jn = (int)(t / g.px) - GH;
    long long src = data_src(g, I, Jn);
    double iJ = 1.0 / J[src];
    double U[8], w[8], Z;
#pragma unroll
    for (int a = 0; a < 8; ++a) U[a] = cons[a * g.N + src] * iJ;
    int st = 0;
    if (inflow && ((g.bc0 == 2 && I < 0) || (g.bc1 == 2 && Jn < 0))) {
        // a ghost beyond an inflow end: the given state
        for (int a = 0; a < 8; ++a) w[a] = inflow[a];
        Z = 0.0;
    } else {
        st = cons2prim_mhd(gam, U, zg_in ? zg_in[src] : -1.0, w, Z);
    }
    bool interior = I >= 0 && I < g.nx && Jn >= 0 && Jn < g.ny;
    if (interior) {
        if (st) atomicAdd(status, 1);
        if (zg_out) zg_out[src] = Z;
    }
    double W = 1.0 / sqrt(1.0 - (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]));
    double beta = w[0] / w[4];
    q[Q_RHO * g.P + t] = w[0];
    q[Q_P * g.P + t] = w[4];
    q[Q_BETA * g.P + t] = beta;
    q[Q_UX * g.P + t] = W * w[1];
    q[Q_UY * g.P + t] = W * w[2];
    q[QM_UZ * g.P + t] = W * w[3];
    q[Q_W * g.P + t] = W;
    // (f32_logs: the mixed form's scheme passes, where the logarithms enter
    // only FP32 arithmetic and the log mean's jump outside its near-equal
    // branch)
    q[Q_LNR * g.P + t] = f32_logs ? f2d_int(logf(d2f_int(w[0]))) : log(w[0]);
    q[Q_LNB * g.P + t] = f32_logs ? f2d_int(logf(d2f_int(beta))) : log(beta);
    q[QM_B1 * g.P + t] = w[5];
    q[QM_B2 * g.P + t] = w[6];
    q[QM_B3 * g.P + t] = w[7];
    double dxi_x = 0.0, dxi_y = 0.0, deta_x = 0.0, deta_y = 0.0;
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        const double a = 0.5 * (P == 1 ? 1.0 : (P == 2 ? (n == 1 ? 4.0 / 3.0 : -1.0 / 6.0)
                                                        : (n == 1 ? 1.5 : (n == 2 ? -0.3 : 1.0 / 30.0))));
        dxi_x += a * (mesh_at(g, x, I + n, Jn, 0, 1) - mesh_at(g, x, I - n, Jn, 0, 1));
        dxi_y += a * (mesh_at(g, x, I + n, Jn, 1, 1) - mesh_at(g, x, I - n, Jn, 1, 1));
        deta_x += a * (mesh_at(g, x, I, Jn + n, 0, 1) - mesh_at(g, x, I, Jn - n, 0, 1));
        deta_y += a * (mesh_at(g, x, I, Jn + n, 1, 1) - mesh_at(g, x, I, Jn - n, 1, 1));
    }
    double M00 = deta_y, M01 = -deta_x, M10 = -dxi_y, M11 = dxi_x;
    q[Q_M00 * g.P + t] = M00;
    q[Q_M01 * g.P + t] = M01;
    q[Q_M10 * g.P + t] = M10;
    q[Q_M11 * g.P + t] = M11;
    double xd = 0.0, yd = 0.0;
    if (xdot) { xd = mesh_at(g, xdot, I, Jn, 0, 0); yd = mesh_at(g, xdot, I, Jn, 1, 0); }
    q[Q_MT0 * g.P + t] = -(xd * M00 + yd * M01);
    q[Q_MT1 * g.P + t] = -(xd * M10 + yd * M11);
}

// entropy variables of a node from its stored values: V = (Gamma/(Gamma-1) +
// ln rho + ln beta/(Gamma-1) + beta, beta u, -beta W, beta b)
template <typename R>
__device__ __forceinline__ void node_V_mhd(const double *__restrict__ q, long long P, long long c, R c1g, R ig,
                                           R V[8])
{
    R beta = (R)q[Q_BETA * P + c], W = (R)q[Q_W * P + c];
    R u0 = (R)q[Q_UX * P + c], u1 = (R)q[Q_UY * P + c], u2 = (R)q[QM_UZ * P + c];
    R B0 = (R)q[QM_B1 * P + c], B1 = (R)q[QM_B2 * P + c], B2 = (R)q[QM_B3 * P + c];
    R b0 = u0 * B0 + u1 * B1 + u2 * B2;
    R bW = beta * rcp<R>(W);
    V[0] = c1g + (R)q[Q_LNR * P + c] + ig * (R)q[Q_LNB * P + c] + beta;
    V[1] = beta * u0;
    V[2] = beta * u1;
    V[3] = beta * u2;
    V[4] = -beta * W;
    V[5] = bW * (B0 + b0 * u0);
    V[6] = bW * (B1 + b0 * u1);
    V[7] = bW * (B2 + b0 * u2);
}

// ES interface flux (eq. ESFlux_HO) between node L in [-1, n_dir - 1] and
// L + 1: the 2p-th order EC sum of two-point fluxes (eq. ECFlux_O2p, summed
// directly), the metric flux (eq. MetricsFlux_O2p), the magnetic flux B~
// (eqs. BFlux_O2p / BFlux_O2) and the WENO dissipation on scaled entropy
// variables at the interface state rho = {{rho}}^ln, u = {{u}},
// p = {{rho}}/{{beta}}, B = {{B}}.
template <typename R, int P, int WW>
__global__ void __launch_bounds__(128) k_iface_mhd(ProbArg pa, Phys ph, const double *__restrict__ q,
                                                   R *__restrict__ iflux, int dir)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    const int nd = dir == 0 ? g.nx : g.ny, no = dir == 0 ? g.ny : g.nx;
    const long long count = (long long)(nd + 1) * no;
    const long long idx = lb * blockDim.x + threadIdx.x;
    if (idx >= count) return;
    int i, j;
    if (dir == 0) { j = (int)(idx / (nd + 1)); i = (int)(idx % (nd + 1)) - 1; }
    else { i = (int)(idx % no); j = (int)(idx / no) - 1; }
    const long long c0 = pidx(g, i, j);
    const long long sd = dir == 0 ? 1 : g.px;
    const double *Mt = q + (Q_MT0 + dir) * g.P;
    const double *Mx = q + (Q_M00 + 2 * dir) * g.P;
    const double *My = q + (Q_M01 + 2 * dir) * g.P;
    const double *B1 = q + QM_B1 * g.P, *B2 = q + QM_B2 * g.P;
    const R gm1inv = (R)(1.0 / (ph.gamma - 1.0));

    R F[8] = {(R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0};
    double Ft = 0.0, Bt = 0.0;
    // (rolled in FP32, for instruction fetch, as in each_index)
#pragma unroll (sizeof(R) == 4 ? 1 : P)
    for (int n = 1; n <= P; ++n) {
        R Fs[8] = {(R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0, (R)0};
        double Fts = 0.0, Bts = 0.0;
#pragma unroll (sizeof(R) == 4 ? 1 : P)
        for (int s = 0; s < n; ++s) {
            const long long cl = c0 - s * sd, cr = cl + n * sd;
            NodeMT<R> l = load_node_m<R>(q, g.P, cl), r = load_node_m<R>(q, g.P, cr);
            R out[8];
            const R mm[3] = {(R)(0.5 * (Mx[cl] + Mx[cr])), (R)(0.5 * (My[cl] + My[cr])), (R)0};
            ec_pair_mhd<2, R>(l, r, gm1inv, ph.ln_thr, (R)(0.5 * (Mt[cl] + Mt[cr])), mm, out);
#pragma unroll
            for (int a = 0; a < 8; ++a) Fs[a] += out[a];
            Fts += 0.5 * (Mt[cl] + Mt[cr]);
            Bts += 0.25 * (Mx[cl] + Mx[cr]) * (B1[cl] + B1[cr]) + 0.25 * (My[cl] + My[cr]) * (B2[cl] + B2[cr]);
        }
        const R an = (R)ph.alpha[n - 1];
#pragma unroll
        for (int a = 0; a < 8; ++a) F[a] += an * Fs[a];
        Ft += ph.alpha[n - 1] * Fts;
        Bt += ph.alpha[n - 1] * Bts;
    }

    if (WW > 0) {
        constexpr int NS = WW + 1, OFF = (WW - 1) / 2;
        const R half = (R)0.5;
        const long long c1 = c0 + sd;
        const R nvx = (R)(0.5 * (Mx[c0] + Mx[c1])), nvy = (R)(0.5 * (My[c0] + My[c1]));
        const R jt = (R)(0.5 * (Mt[c0] + Mt[c1]));
        const R Lk = sq_rt<R>(nvx * nvx + nvy * nvy);
        const R iLk = rcp<R>(Lk), nx = nvx * iLk, ny = nvy * iLk;
        // interface state
        R wm[8], wrot[8];
        {
            R rho, irho;
            lmean<R, double>(q[Q_RHO * g.P + c0], q[Q_RHO * g.P + c1], q[Q_LNR * g.P + c0], q[Q_LNR * g.P + c1],
                             (R)q[Q_RHO * g.P + c0], (R)q[Q_RHO * g.P + c1], ph.ln_thr, rho, irho);
            R um[3] = {half * ((R)q[Q_UX * g.P + c0] + (R)q[Q_UX * g.P + c1]),
                       half * ((R)q[Q_UY * g.P + c0] + (R)q[Q_UY * g.P + c1]),
                       half * ((R)q[QM_UZ * g.P + c0] + (R)q[QM_UZ * g.P + c1])};
            R W2 = (R)1 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
            R W = sq_rt<R>(W2);
            wm[0] = rho;
            const R iW = rcp<R>(W);
            for (int k = 0; k < 3; ++k) wm[1 + k] = um[k] * iW;
            wm[4] = ((R)q[Q_RHO * g.P + c0] + (R)q[Q_RHO * g.P + c1]) *
                    rcp<R>((R)q[Q_BETA * g.P + c0] + (R)q[Q_BETA * g.P + c1]);
            wm[5] = half * ((R)B1[c0] + (R)B1[c1]);
            wm[6] = half * ((R)B2[c0] + (R)B2[c1]);
            wm[7] = half * ((R)q[QM_B3 * g.P + c0] + (R)q[QM_B3 * g.P + c1]);
            wrot[0] = wm[0];
            wrot[1] = nx * wm[1] + ny * wm[2];
            wrot[2] = -ny * wm[1] + nx * wm[2];
            wrot[3] = wm[3];
            wrot[4] = wm[4];
            wrot[5] = nx * wm[5] + ny * wm[6];
            wrot[6] = -ny * wm[5] + nx * wm[6];
            wrot[7] = wm[7];
        }
        R lam[8], Rm[8][8];
        eigen_mhd<R>(ph.gamma, wrot, lam, Rm, true);
        R lhat = (R)0;
#pragma unroll
        for (int m = 0; m < 8; ++m) lhat = vmax(lhat, fab<R>(jt + Lk * lam[m]));
        const R ig = gm1inv, c1g = (R)ph.gamma * gm1inv;
        R Vt[NS][8], scale[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) scale[m] = (R)0;
        for (int k = 0; k < NS; ++k) {
            R V[8], TV[8];
            node_V_mhd<R>(q, g.P, c0 + (k - OFF) * sd, c1g, ig, V);
            TV[0] = V[0];
            TV[1] = nx * V[1] + ny * V[2];
            TV[2] = -ny * V[1] + nx * V[2];
            TV[3] = V[3];
            TV[4] = V[4];
            TV[5] = nx * V[5] + ny * V[6];
            TV[6] = -ny * V[5] + nx * V[6];
            TV[7] = V[7];
            for (int m = 0; m < 8; ++m) {
                R acc = (R)0;
                for (int a = 0; a < 8; ++a) {
                    R t = Rm[a][m] * TV[a];
                    acc += t;
                    if (k == OFF || k == OFF + 1) scale[m] += fab<R>(t);
                }
                Vt[k][m] = acc;
            }
        }
        R z[8];
        const R eps = (R)ph.eps, sign_tol = (R)ph.sign_tol;
        each_index<R>(8, [&](int m) {
            R vminus, vplus;
            if (WW == 5)
                weno5_lr<R>(Vt[0][m], Vt[1][m], Vt[2][m], Vt[3][m], Vt[4][m], Vt[5][m], eps, vminus, vplus);
            else
                weno3_lr<R>(Vt[0][m], Vt[1][m], Vt[2][m], Vt[3][m], eps, vminus, vplus);
            R jw = vplus - vminus;
            R jump = Vt[OFF + 1][m] - Vt[OFF][m];
            int sj = le(fab<R>(jump), sign_tol * scale[m]) ? 0 : sgn_d(jump);
            z[m] = (sgn_d(jw) == sj) ? jw : (R)0;
        });
        R d[8];
        for (int a = 0; a < 8; ++a) {
            R acc = (R)0;
            for (int m = 0; m < 8; ++m) acc += Rm[a][m] * z[m];
            d[a] = acc;
        }
        const R hl = half * lhat;
        F[0] -= hl * d[0];
        F[1] -= hl * (nx * d[1] - ny * d[2]);
        F[2] -= hl * (ny * d[1] + nx * d[2]);
        F[3] -= hl * d[3];
        F[4] -= hl * d[4];
        F[5] -= hl * (nx * d[5] - ny * d[6]);
        F[6] -= hl * (ny * d[5] + nx * d[6]);
        F[7] -= hl * d[7];
    }
    R *out = iflux + (long long)(dir * NFM) * g.P + c0;
#pragma unroll
    for (int a = 0; a < 8; ++a) out[a * g.P] = F[a];
    out[8 * g.P] = (R)Ft;
    out[9 * g.P] = (R)Bt;
}

// initial J and cons = J U(prim)
template <int P>
__global__ void k_init_state_mhd(ProbArg pa, double gam, const double *__restrict__ prim,
                                 const double *__restrict__ x, double *__restrict__ cons, double *__restrict__ J,
                                 int *status)
{
    ProbDesc D;
    long long lb;
    locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    double dxi_x = 0.0, dxi_y = 0.0, deta_x = 0.0, deta_y = 0.0;
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        const double a = 0.5 * (P == 1 ? 1.0 : (P == 2 ? (n == 1 ? 4.0 / 3.0 : -1.0 / 6.0)
                                                        : (n == 1 ? 1.5 : (n == 2 ? -0.3 : 1.0 / 30.0))));
        dxi_x += a * (mesh_at(g, x, i + n, j, 0, 1) - mesh_at(g, x, i - n, j, 0, 1));
        dxi_y += a * (mesh_at(g, x, i + n, j, 1, 1) - mesh_at(g, x, i - n, j, 1, 1));
        deta_x += a * (mesh_at(g, x, i, j + n, 0, 1) - mesh_at(g, x, i, j - n, 0, 1));
        deta_y += a * (mesh_at(g, x, i, j + n, 1, 1) - mesh_at(g, x, i, j - n, 1, 1));
    }
    double J0 = dxi_x * deta_y - deta_x * dxi_y;
    double w[8], U[8], F[8], V[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) w[a] = prim[a * g.N + id];
    double v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
    if (!(w[0] > 0.0) || !(w[4] > 0.0) || !(v2 < 1.0) || !(J0 > 0.0)) {
        atomicAdd(status + 1, 1);
        w[0] = 1.0; w[4] = 1.0; w[1] = w[2] = w[3] = 0.0;   // keep the arithmetic finite
    }
    mhd_UFV<double>(gam, w, U, F, V);
    J[id] = J0;
#pragma unroll
    for (int a = 0; a < 8; ++a) cons[a * g.N + id] = J0 * U[a];
}

// d/dt = -sum_k (F_k(i+1/2) - F_k(i-1/2)) - Phi'(V_i) sum_k (B~_k(i+1/2) -
// B~_k(i-1/2)) (eq. RMHDSemiU_O2p_ES), dJ/dt from the metric flux; written
// out (dcons != NULL) or combined into the SSP-RK3 stage as in k_update.
template <typename R>
__global__ void k_update_mhd(ProbArg pa, const double *__restrict__ q, const R *__restrict__ fl,
                             double *__restrict__ dcons, double *__restrict__ dJ, const double *__restrict__ cn,
                             const double *__restrict__ Jn_, const double *__restrict__ xn,
                             const double *__restrict__ cs, const double *__restrict__ Js,
                             const double *__restrict__ xs, const double *__restrict__ xdot, double A, double B,
                             const double *__restrict__ dt_dev, double *__restrict__ co, double *__restrict__ Jo,
                             double *__restrict__ xo)
{
    ProbDesc D;
    long long lb;
    int b = locate(pa, D, lb);
    const Geom &g = D.g;
    long long id = lb * blockDim.x + threadIdx.x;
    if (id >= g.N) return;
    int i = (int)(id % g.nx), j = (int)(id / g.nx);
    long long c = pidx(g, i, j);
    const R *f0 = fl, *f1 = fl + NFM * g.P;
    double L[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) {
        double d0 = to_f64(f0[a * g.P + c]) - to_f64(f0[a * g.P + c - 1]);
        double d1 = to_f64(f1[a * g.P + c]) - to_f64(f1[a * g.P + c - g.px]);
        L[a] = -(d0 + d1);
    }
    // Powell source: L[9] = -div B~ here
    double iW = 1.0 / q[Q_W * g.P + c];
    double w[8];
    w[1] = q[Q_UX * g.P + c] * iW;
    w[2] = q[Q_UY * g.P + c] * iW;
    w[3] = q[QM_UZ * g.P + c] * iW;
    w[5] = q[QM_B1 * g.P + c];
    w[6] = q[QM_B2 * g.P + c];
    w[7] = q[QM_B3 * g.P + c];
    double Pp[8];
    mhd_phiprime(w, Pp);
#pragma unroll
    for (int a = 0; a < 8; ++a) L[a] += Pp[a] * L[9];
    if (dcons) {
#pragma unroll
        for (int a = 0; a < 8; ++a) dcons[a * g.N + id] = L[a];
        dJ[id] = L[8];
        return;
    }
    double dt = dt_dev[b];
#pragma unroll
    for (int a = 0; a < 8; ++a) co[a * g.N + id] = A * cn[a * g.N + id] + B * (cs[a * g.N + id] + dt * L[a]);
    Jo[id] = A * Jn_[id] + B * (Js[id] + dt * L[8]);
    xo[id] = A * xn[id] + B * (xs[id] + dt * xdot[id]);
    xo[g.N + id] = A * xn[g.N + id] + B * (xs[g.N + id] + dt * xdot[g.N + id]);
}


template <typename R, int P>
static void launch_iface_mhd_p(const LaunchDom &L, const Phys &ph, const double *q, R *iflux, int dir, cudaStream_t st)
{
    switch (ph.w) {
    case 0: k_iface_mhd<R, P, 0><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, iflux, dir); break;
    case 3: k_iface_mhd<R, P, 3><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, iflux, dir); break;
    default: k_iface_mhd<R, P, 5><<<L.nblk, L.bs, 0, st>>>(L.pa, ph, q, iflux, dir); break;
    }
}

// interface fluxes of one sweep direction in the working precision R
template <typename R>
static void launch_iface_mhd_t(const LaunchDom &L, const Phys &ph, const double *q, void *iflux, int dir,
                               cudaStream_t st)
{
    R *fl = (R *)iflux;
    switch (ph.p) {
    case 1: launch_iface_mhd_p<R, 1>(L, ph, q, fl, dir, st); break;
    case 2: launch_iface_mhd_p<R, 2>(L, ph, q, fl, dir, st); break;
    default: launch_iface_mhd_p<R, 3>(L, ph, q, fl, dir, st); break;
    }
}

template <typename R>
static void launch_update_mhd_t(const LaunchDom &L, const double *q, const void *fl, double *dcons, double *dJ,
                                const double *cn, const double *Jn, const double *xn, const double *cs,
                                const double *Js, const double *xs, const double *xdot, double A, double B,
                                const double *dt_dev, double *co, double *Jo, double *xo, cudaStream_t st)
{
    k_update_mhd<R><<<L.nblk, L.bs, 0, st>>>(L.pa, q, (const R *)fl, dcons, dJ, cn, Jn, xn, cs, Js, xs, xdot, A, B,
                                             dt_dev, co, Jo, xo);
}

}  // namespace esmm
