// esmm_device.cuh -- device arithmetic of the ES adaptive moving-mesh scheme
// (Duan & Tang, arXiv 2107.12027), 2D RHD, templated on the working precision
// R (double for the FP64 form, float for the mixed form).  The primitive
// recovery is always FP64, and so are the jumps of the logarithmic mean.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "esmm_conv.h"

namespace esmm {

constexpr int GH = 3;        // ghost layers of the padded node arrays
constexpr int PMAX = 3;      // largest supported p
// Node quantities stored per padded node (FP64, structure of arrays).
enum {
    Q_RHO = 0, Q_P, Q_BETA, Q_UX, Q_UY, Q_W, Q_LNR, Q_LNB,
    Q_M00, Q_M01, Q_M10, Q_M11, Q_MT0, Q_MT1, NQ
};
// FP32 copies of the node quantities that the mixed form's flux kernels read
// (written by the FP64 node pass, so that no flux kernel converts a double).
enum {
    Q32_R = 0, Q32_B, Q32_UX, Q32_UY, Q32_W, Q32_LNR, Q32_LNB,
    Q32_M00, Q32_M01, Q32_M10, Q32_M11, Q32_MT0, Q32_MT1, NQ32
};

struct Geom {
    int nx, ny;       // interior nodes
    int px, py;       // padded extents nx + 2 GH, ny + 2 GH
    long long P;      // px * py
    long long N;      // nx * ny
    int bc0, bc1;     // 0 periodic, 1 outflow
    double per0, per1;
    int own0, own1;   // rows j in [own0, own1) take part in the reductions
                      // (0, ny except on a slab of a decomposed grid)
};

// a node in the rows whose values the problem's reductions collect
__device__ __forceinline__ bool owned_row(const Geom &g, int j) { return j >= g.own0 && j < g.own1; }

// One problem of a batch: its geometry and the offsets of its slices in the
// concatenated arrays (on: node arrays, in units of nodes; op: padded-node
// arrays, in units of padded nodes).
struct ProbDesc {
    Geom g;
    long long on, op;
};

// Problem addressing of a launch: a single problem passed by value (tiles ==
// nullptr), or a device table of problems with a map from block to
// (problem, block within the problem), so that no block spans two problems.
struct ProbArg {
    const ProbDesc *pd;
    const int2 *tiles;
    ProbDesc one;
};

__device__ __forceinline__ int locate(const ProbArg &pa, ProbDesc &D, long long &local_block)
{
    if (pa.tiles) {
        int2 t = pa.tiles[blockIdx.x];
        D = pa.pd[t.x];
        local_block = t.y;
        return t.x;
    }
    D = pa.one;
    local_block = blockIdx.x;
    return 0;
}

// locate() for tile t of a strided launch (the block -> tile map of a
// batch, or tile t itself)
__device__ __forceinline__ int locate_tile(const ProbArg &pa, long long t, ProbDesc &D, long long &local_block)
{
    if (pa.tiles) {
        int2 tt = pa.tiles[t];
        D = pa.pd[tt.x];
        local_block = tt.y;
        return tt.x;
    }
    D = pa.one;
    local_block = t;
    return 0;
}

// The site (i, j) of thread threadIdx.x in tile lb of a sweep of direction
// dir over sites with ext extra positions before the first node along the
// sweep (p node pairs, 1 interface).  tx = 0: tiles are flat runs along the
// sweep's storage order; tx > 0: tiles of tx sites along x_1 by
// blockDim.x / tx along x_2.  false: no site (ragged tile).
__device__ __forceinline__ bool sweep_site(const Geom &g, int dir, int ext, int tx, long long lb, int &i, int &j)
{
    const int nd = dir == 0 ? g.nx : g.ny, no = dir == 0 ? g.ny : g.nx;
    if (tx == 0) {
        const long long idx = lb * blockDim.x + threadIdx.x;
        if (idx >= (long long)(nd + ext) * no) return false;
        if (dir == 0) { j = (int)(idx / (nd + ext)); i = (int)(idx % (nd + ext)) - ext; }
        else { i = (int)(idx % no); j = (int)(idx / no) - ext; }
        return true;
    }
    const int ty = blockDim.x / tx;
    const int Ei = dir == 0 ? nd + ext : no, Ej = dir == 0 ? no : nd + ext;
    const long long nbi = (Ei + tx - 1) / tx;
    const int ii = (int)(lb % nbi) * tx + (int)threadIdx.x % tx;
    const int jj = (int)(lb / nbi) * ty + (int)threadIdx.x / tx;
    if (ii >= Ei || jj >= Ej) return false;
    i = dir == 0 ? ii - ext : ii;
    j = dir == 0 ? jj : jj - ext;
    return true;
}

// FP64 <-> FP32 conversions on the integer pipes (esmm_conv.h), equal bit
// for bit to the hardware conversions, which issue on the FP64 pipe
template <typename T>
__device__ __forceinline__ T from_f64(double x);
template <>
__device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_f64<float>(double x) { return d2f_int(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f2d_int(x); }

struct Phys {
    double gamma;
    double gm1i;      // 1 / (Gamma - 1), once per launch
    double eps;       // WENO epsilon
    double ln_thr;    // log-mean series switch on ((b-a)/(b+a))^2
    double sign_tol;  // relative size below which [[V~]] counts as zero
    double alpha[PMAX];
    int p, w;
};

__host__ __device__ __forceinline__ long long pidx(const Geom &g, int i, int j)
{
    return (long long)(j + GH) * g.px + (i + GH);
}

__device__ __forceinline__ int wrapi(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }
__device__ __forceinline__ int floordivi(int a, int n) { return a >= 0 ? a / n : -((-a + n - 1) / n); }
__device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

// Boundary data: periodic wrap or zero-gradient copy.
__device__ __forceinline__ long long data_src(const Geom &g, int i, int j)
{
    int ii = g.bc0 == 0 ? wrapi(i, g.nx) : clampi(i, 0, g.nx - 1);
    int jj = g.bc1 == 0 ? wrapi(j, g.ny) : clampi(j, 0, g.ny - 1);
    return (long long)jj * g.nx + ii;
}

// Boundary mesh: periodic wrap plus the period (shift = 1 for coordinates,
// 0 for velocities), or linear extrapolation of the two boundary nodes.
__device__ __forceinline__ double mesh_along_i(const Geom &g, const double *a, int i, int j, int comp, int shift)
{
    const double *row = a + (long long)comp * g.N + (long long)j * g.nx;
    if (g.bc0 == 0) {
        double s = (shift && comp == 0) ? floordivi(i, g.nx) * g.per0 : 0.0;
        return row[wrapi(i, g.nx)] + s;
    }
    if (i < 0) { double a0 = row[0], a1 = row[1]; return a0 + i * (a1 - a0); }
    if (i >= g.nx) { double a0 = row[g.nx - 1], a1 = row[g.nx - 2]; return a0 + (i - (g.nx - 1)) * (a0 - a1); }
    return row[i];
}

__device__ __forceinline__ double mesh_at(const Geom &g, const double *a, int i, int j, int comp, int shift)
{
    if (g.bc1 == 0) {
        double s = (shift && comp == 1) ? floordivi(j, g.ny) * g.per1 : 0.0;
        return mesh_along_i(g, a, i, wrapi(j, g.ny), comp, shift) + s;
    }
    if (j < 0) {
        double a0 = mesh_along_i(g, a, i, 0, comp, shift), a1 = mesh_along_i(g, a, i, 1, comp, shift);
        return a0 + j * (a1 - a0);
    }
    if (j >= g.ny) {
        double a0 = mesh_along_i(g, a, i, g.ny - 1, comp, shift), a1 = mesh_along_i(g, a, i, g.ny - 2, comp, shift);
        return a0 + (j - (g.ny - 1)) * (a0 - a1);
    }
    return mesh_along_i(g, a, i, j, comp, shift);
}

// ---------------------------------------------------------------------------
// Conservative -> primitive recovery (FP64 in every form).  Newton on p for
//   f(p) = (G-1)/G ((E+p)(1-v^2) - D sqrt(1-v^2)) - p,  v = |m|/(E+p),
// safeguarded by bisection on [0, (G-1)E], stopping when a step moves p by at
// most 1e-15 (E + p), the resolution of E + p from which f is evaluated, or
// when |f| <= 2e-15 (E + p), f's own rounding level (where df/dp is small,
// steps at that level exceed the first bound and the loop would bisect);
// p0 is a warm start (ignored when outside the bracket).  The Newton step
// divides by df through an FP32 reciprocal: the slope only steers the step
// (a relative slope error e contracts the error by e per step), while f, which
// decides the stopping, is FP64.  W receives the Lorentz factor 1/sqrt(1-v^2)
// (1 for a non-admissible state).  Returns 0, 1 for a non-admissible state, 2
// when the iteration cap is hit.  gg = (Gamma - 1)/Gamma, which a launch can
// pass in (one division per launch, not per node).
__device__ __forceinline__ int cons2prim_gg(double gam, double gg, double D, double mx, double my, double E,
                                            double p0, double &rho, double &vx, double &vy, double &p, double &W)
{
    double S2 = mx * mx + my * my;
    double S = sqrt(S2);
    rho = 0.0; vx = 0.0; vy = 0.0; p = 0.0; W = 1.0;
    if (!(D > 0.0) || !(E * E > D * D + S2) || !(E > 0.0)) return 1;
    double lo = 0.0, hi = (gam - 1.0) * E;
    double pc = (p0 > lo && p0 < hi) ? p0 : 0.5 * (lo + hi);
    int ok = 0;
    bool have = false;        // r, iW2, rs below belong to pc
    double r = 0.0, iW2 = 0.0, rs = 0.0;
    for (int it = 0; it < 200; ++it) {
        double Ep = E + pc;
        r = __drcp_rn(Ep);
        iW2 = (Ep - S) * (Ep + S) * r * r;           // 1 - v^2
        rs = rsqrt(iW2);
        double iW = iW2 * rs;                        // sqrt(1 - v^2)
        double v2 = S2 * r * r;
        double f = gg * (Ep * iW2 - D * iW) - pc;
        double df = gg * (1.0 + v2 - D * v2 * r * rs) - 1.0;
        if (fabs(f) <= 2.0e-15 * (E + pc)) { ok = 1; have = true; break; }   // residual at rounding level
        double pn = pc;                              // f = 0: pc is a root
        if (f != 0.0) {
            if (f > 0.0) lo = pc; else hi = pc;
            pn = pc - f * f2d_int(__frcp_rn(d2f_int(df)));
            if (!(pn > lo && pn < hi)) pn = 0.5 * (lo + hi);
        }
        if (fabs(pn - pc) <= 1.0e-15 * (E + pn)) { have = pn == pc; pc = pn; ok = 1; break; }
        pc = pn;
    }
    if (!have) {
        double Ep = E + pc;
        r = __drcp_rn(Ep);
        iW2 = (Ep - S) * (Ep + S) * r * r;
        rs = rsqrt(iW2);
    }
    rho = D * (iW2 * rs);
    vx = mx * r;
    vy = my * r;
    p = pc;
    W = rs;
    return ok ? 0 : 2;
}

__device__ __forceinline__ int cons2prim(double gam, double D, double mx, double my, double E,
                                         double p0, double &rho, double &vx, double &vy, double &p, double &W)
{
    return cons2prim_gg(gam, (gam - 1.0) / gam, D, mx, my, E, p0, rho, vx, vy, p, W);
}

// ---------------------------------------------------------------------------
// Dual number a + b eps (eps^2 = 0): the flux arithmetic below is templated on
// its working type, and evaluating it on duals seeded at one input gives the
// derivative of every output with respect to that input.  The adjoint kernels
// use this for the local (per pair / per interface) Jacobian-vector products.
struct dual {
    double v, d;
    __host__ __device__ dual() {}
    __host__ __device__ constexpr dual(double a) : v(a), d(0.0) {}
    __host__ __device__ constexpr dual(double a, double b) : v(a), d(b) {}
};
__device__ __forceinline__ dual operator+(dual a, dual b) { return dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ dual operator-(dual a, dual b) { return dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ dual operator-(dual a) { return dual(-a.v, -a.d); }
__device__ __forceinline__ dual operator*(dual a, dual b) { return dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ dual operator/(dual a, dual b)
{
    double r = __drcp_rn(b.v);
    double q = a.v * r;
    return dual(q, (a.d - q * b.d) * r);
}
__device__ __forceinline__ dual operator+(dual a, double b) { return dual(a.v + b, a.d); }
__device__ __forceinline__ dual operator+(double a, dual b) { return dual(a + b.v, b.d); }
__device__ __forceinline__ dual operator-(dual a, double b) { return dual(a.v - b, a.d); }
__device__ __forceinline__ dual operator-(double a, dual b) { return dual(a - b.v, -b.d); }
__device__ __forceinline__ dual operator*(dual a, double b) { return dual(a.v * b, a.d * b); }
__device__ __forceinline__ dual operator*(double a, dual b) { return dual(a * b.v, a * b.d); }
__device__ __forceinline__ dual operator/(dual a, double b)
{
    const double r = __drcp_rn(b);
    return dual(a.v * r, a.d * r);
}
__device__ __forceinline__ dual operator/(double a, dual b) { return dual(a) / b; }
__device__ __forceinline__ dual &operator+=(dual &a, dual b) { a = a + b; return a; }
__device__ __forceinline__ dual &operator-=(dual &a, dual b) { a = a - b; return a; }
__device__ __forceinline__ dual &operator*=(dual &a, dual b) { a = a * b; return a; }
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ float val(float x) { return x; }
__device__ __forceinline__ double val(dual x) { return x.v; }

// The FP32 dual number (directional derivatives inside the FP32 bulk form).
// FP64 constants are rounded to FP32 before they meet an fdual, so no FP64
// arithmetic runs on its values.
struct fdual {
    float v, d;
    __host__ __device__ fdual() {}
    __host__ __device__ constexpr fdual(float a) : v(a), d(0.0f) {}
    __host__ __device__ constexpr fdual(float a, float b) : v(a), d(b) {}
};
__device__ __forceinline__ fdual operator+(fdual a, fdual b) { return fdual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ fdual operator-(fdual a, fdual b) { return fdual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ fdual operator-(fdual a) { return fdual(-a.v, -a.d); }
__device__ __forceinline__ fdual operator*(fdual a, fdual b) { return fdual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ fdual operator/(fdual a, fdual b)
{
    float r = __frcp_rn(b.v);
    float q = a.v * r;
    return fdual(q, (a.d - q * b.d) * r);
}
__device__ __forceinline__ fdual operator+(fdual a, double b) { return fdual(a.v + (float)b, a.d); }
__device__ __forceinline__ fdual operator+(double a, fdual b) { return fdual((float)a + b.v, b.d); }
__device__ __forceinline__ fdual operator-(fdual a, double b) { return fdual(a.v - (float)b, a.d); }
__device__ __forceinline__ fdual operator-(double a, fdual b) { return fdual((float)a - b.v, -b.d); }
__device__ __forceinline__ fdual operator*(fdual a, double b) { return fdual(a.v * (float)b, a.d * (float)b); }
__device__ __forceinline__ fdual operator*(double a, fdual b) { return fdual((float)a * b.v, (float)a * b.d); }
__device__ __forceinline__ fdual operator/(fdual a, double b) { return a / fdual((float)b); }
__device__ __forceinline__ fdual operator/(double a, fdual b) { return fdual((float)a) / b; }
__device__ __forceinline__ fdual &operator+=(fdual &a, fdual b) { a = a + b; return a; }
__device__ __forceinline__ fdual &operator-=(fdual &a, fdual b) { a = a - b; return a; }

// Hyper-dual number v + a e1 + b e2 + ab e1 e2 (e1^2 = e2^2 = 0): e1 carries a
// Jacobian image direction, e2 the adjoint's seeded state direction, and ab
// the mixed second derivative.  Used for the images of the RMHD
// eigen-system inside the adjoint.
struct hdual {
    double v, a, b, ab;
    __host__ __device__ hdual() {}
    __host__ __device__ constexpr hdual(double x) : v(x), a(0.0), b(0.0), ab(0.0) {}
    __host__ __device__ constexpr hdual(double x, double a_, double b_, double ab_) : v(x), a(a_), b(b_), ab(ab_) {}
};
__device__ __forceinline__ hdual operator+(hdual x, hdual y) { return hdual(x.v + y.v, x.a + y.a, x.b + y.b, x.ab + y.ab); }
__device__ __forceinline__ hdual operator-(hdual x, hdual y) { return hdual(x.v - y.v, x.a - y.a, x.b - y.b, x.ab - y.ab); }
__device__ __forceinline__ hdual operator-(hdual x) { return hdual(-x.v, -x.a, -x.b, -x.ab); }
__device__ __forceinline__ hdual operator*(hdual x, hdual y)
{
    return hdual(x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b,
                 x.ab * y.v + x.a * y.b + x.b * y.a + x.v * y.ab);
}
// f(x) for a scalar function with value f, first and second derivatives f1, f2 at x.v
__device__ __forceinline__ hdual hchain(hdual x, double f, double f1, double f2)
{
    return hdual(f, f1 * x.a, f1 * x.b, f1 * x.ab + f2 * x.a * x.b);
}
__device__ __forceinline__ hdual hrcp(hdual x)
{
    double r = __drcp_rn(x.v);
    return hchain(x, r, -r * r, 2.0 * r * r * r);
}
__device__ __forceinline__ hdual operator/(hdual x, hdual y) { return x * hrcp(y); }
__device__ __forceinline__ hdual operator+(hdual x, double y) { return hdual(x.v + y, x.a, x.b, x.ab); }
__device__ __forceinline__ hdual operator+(double x, hdual y) { return hdual(x + y.v, y.a, y.b, y.ab); }
__device__ __forceinline__ hdual operator-(hdual x, double y) { return hdual(x.v - y, x.a, x.b, x.ab); }
__device__ __forceinline__ hdual operator-(double x, hdual y) { return hdual(x - y.v, -y.a, -y.b, -y.ab); }
__device__ __forceinline__ hdual operator*(hdual x, double y) { return hdual(x.v * y, x.a * y, x.b * y, x.ab * y); }
__device__ __forceinline__ hdual operator*(double x, hdual y) { return hdual(x * y.v, x * y.a, x * y.b, x * y.ab); }
__device__ __forceinline__ hdual operator/(hdual x, double y) { return x * __drcp_rn(y); }
__device__ __forceinline__ hdual operator/(double x, hdual y) { return x * hrcp(y); }

// the dual number over a working precision (hdual over dual)
template <typename R> struct DualOf { using type = dual; };
template <> struct DualOf<float> { using type = fdual; };
template <> struct DualOf<dual> { using type = hdual; };
// an image seed: value w moved along direction d (for hdual: w, d are duals
// whose .d parts are the seeded state direction and d's derivative along it)
__device__ __forceinline__ dual img_seed(double w, double d) { return dual(w, d); }
__device__ __forceinline__ fdual img_seed(float w, float d) { return fdual(w, d); }
__device__ __forceinline__ hdual img_seed(dual w, dual d) { return hdual(w.v, d.v, w.d, d.d); }
// the image part of a seeded result, in the working precision
__device__ __forceinline__ double img_part(dual x) { return x.d; }
__device__ __forceinline__ float img_part(fdual x) { return x.d; }
__device__ __forceinline__ dual img_part(hdual x) { return dual(x.a, x.ab); }

// type of the log-mean arguments: FP64 for the FP64 and FP32-bulk forms
template <typename R> struct LogT { using type = double; };
template <> struct LogT<dual> { using type = dual; };

template <typename R> __device__ __forceinline__ R rsq(R x);
template <> __device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ dual rsq<dual>(dual x)
{
    double r = rsqrt(x.v);
    return dual(r, -0.5 * r * r * r * x.d);
}
template <typename R> __device__ __forceinline__ R sq_rt(R x);
template <> __device__ __forceinline__ double sq_rt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float sq_rt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ dual sq_rt<dual>(dual x)
{
    double r = sqrt(x.v);
    return dual(r, 0.5 * x.d / r);
}
template <> __device__ __forceinline__ fdual sq_rt<fdual>(fdual x)
{
    float r = sqrtf(x.v);
    return fdual(r, 0.5f * x.d * __frcp_rn(r));
}
template <> __device__ __forceinline__ hdual sq_rt<hdual>(hdual x)
{
    double r = sqrt(x.v);
    double r1 = 0.5 / r;
    return hchain(x, r, r1, -0.5 * r1 / x.v);
}
// reciprocal (IEEE round-to-nearest) and a square root of a positive value
// through the reciprocal square root: on GB300 both are cheaper than the
// FP64 quotient and square root
template <typename R> __device__ __forceinline__ R rcp(R x);
template <> __device__ __forceinline__ double rcp<double>(double x) { return __drcp_rn(x); }
template <> __device__ __forceinline__ float rcp<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ dual rcp<dual>(dual x)
{
    double r = __drcp_rn(x.v);
    return dual(r, -r * r * x.d);
}
template <> __device__ __forceinline__ fdual rcp<fdual>(fdual x)
{
    float r = __frcp_rn(x.v);
    return fdual(r, -r * r * x.d);
}
template <> __device__ __forceinline__ hdual rcp<hdual>(hdual x) { return hrcp(x); }
template <> __device__ __forceinline__ fdual rsq<fdual>(fdual x)
{
    float r = rsqrtf(x.v);
    return fdual(r, -0.5f * r * r * r * x.d);
}
template <> __device__ __forceinline__ hdual rsq<hdual>(hdual x)
{
    // x^-1/2 and its first two derivatives
    double r = rsqrt(x.v), ir = __drcp_rn(x.v);
    return hchain(x, r, -0.5 * r * ir, 0.75 * r * ir * ir);
}
template <typename R> __device__ __forceinline__ R sqrt_pos(R x) { return x * rsq<R>(x); }
template <typename R> __device__ __forceinline__ R fab(R x);
template <> __device__ __forceinline__ double fab<double>(double x) { return fabs(x); }
template <> __device__ __forceinline__ float fab<float>(float x) { return fabsf(x); }
template <> __device__ __forceinline__ dual fab<dual>(dual x) { return x.v < 0.0 ? -x : x; }
// larger of two values (the derivative follows the selected argument)
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ dual vmax(dual a, dual b) { return a.v >= b.v ? a : b; }

// Logarithmic mean [[a]]/[[ln a]] and its reciprocal from FP64 node values
// and their FP64 logarithms.  Near-equal arguments, ((b-a)/(b+a))^2 < thr, use
// the Ismail-Roe series in FP64: mean = (a+b)/(2 F), F = 1 + u/3 + u^2/5 + u^3/7.
template <typename R, typename T>
__device__ __forceinline__ void logmean(T a, T b, T la, T lb, double thr, R &mean, R &inv_mean)
{
    T d = b - a, s = b + a;
    if (val(d * d) < val(thr * s * s)) {
        // (two reciprocals for the three quotients: each product is within
        // an ulp of the quotient it stands for)
        T is = rcp<T>(s);
        T r = d * is, u = r * r;
        T F = 1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0)));
        mean = (R)(0.5 * s * rcp<T>(F));
        inv_mean = (R)(2.0 * F * is);
    } else {
        R dn = (R)d, dl = (R)(lb - la);
        mean = dn * rcp<R>(dl);
        inv_mean = dl * rcp<R>(dn);
    }
}

// The log mean of two nodes, a32 and b32 being the working-precision copies
// of a and b: in FP64 and on duals exactly logmean.  In FP32 the jumps b - a
// and ln b - ln a, which cancel at near-equal states, are taken in FP64 from
// the FP64 node values; the series (switch at (b-a)^2 < thr (a+b)^2) and the
// quotients then run in FP32, whose rounding of the result they already are
// below (the series' terms beyond 1 are < thr/3).
template <typename R, typename T>
__device__ __forceinline__ void lmean(T a, T b, T la, T lb, R a32, R b32, double thr, R &mean, R &inv_mean)
{
    logmean<R, T>(a, b, la, lb, thr, mean, inv_mean);
}
template <>
__device__ __forceinline__ void lmean<float, double>(double a, double b, double la, double lb, float a32, float b32,
                                                     double thr, float &mean, float &inv_mean)
{
    const float d = (float)(b - a), s = a32 + b32;
    if (d * d < (float)thr * (s * s)) {
        const float is = __frcp_rn(s);
        const float r = d * is, u = r * r;
        const float F = 1.0f + u * (1.0f / 3.0f + u * (1.0f / 5.0f + u * (1.0f / 7.0f)));
        mean = 0.5f * s * __frcp_rn(F);
        inv_mean = 2.0f * F * is;
    } else {
        const float dl = (float)(lb - la);
        mean = d * __frcp_rn(dl);
        inv_mean = dl * __frcp_rn(d);
    }
}

// Node values of one two-point flux argument (the parameter variables).
template <typename R>
struct NodeV {
    typename LogT<R>::type rho, beta, lnr, lnb;  // log-mean arguments (FP64 unless dual)
    R r, b, ux, uy, W;
};

// Curvilinear two-point EC flux of Sec. 3.1 for one node pair in direction k:
//   F~_k = 1/2 (mt_l + mt_r) U~ + sum_j 1/2 (M_kj,l + M_kj,r) F~_j,
// mt, mx, my the averaged metrics.  U~ is the paper's U~^RMHD at B = 0 and
// F~_j the matching RHD spatial flux:
//   U~_D = r_ln W,  U~_E = (alpha0 U~_D W + pm |u|^2)/Lam,
//   U~_m = (U~_E + pm) u/W,  F~_D,j = r_ln u_j,
//   F~_E,j = W (alpha0 r_ln + pm) u_j / Lam,  F~_m,j = F~_E,j u/W + pm e_j,
// with the arithmetic means r, b, u, W, pm = r/b, Lam = W^2 - |u|^2 and
// alpha0 = 1 + 1/((Gamma-1) b_ln).  Contracting with the metrics gives
//   out_D = r_ln (mt W + un), out_E = mt U~_E + Es,
//   out_m = u/W (mt (U~_E + pm) + Es) + pm (mx, my),
// un = mx u_x + my u_y, Es = W (alpha0 r_ln + pm) un / Lam.
template <typename R>
__device__ __forceinline__ void ec_pair(const NodeV<R> &l, const NodeV<R> &r, R mt, R mx, R my,
                                        R gm1inv, double thr, R out[4])
{
    R rln, irln, bln, ibln;
    lmean<R, typename LogT<R>::type>(l.rho, r.rho, l.lnr, r.lnr, l.r, r.r, thr, rln, irln);
    lmean<R, typename LogT<R>::type>(l.beta, r.beta, l.lnb, r.lnb, l.b, r.b, thr, bln, ibln);
    R half = (R)0.5;
    R rm = half * (l.r + r.r);
    R bm = half * (l.b + r.b);
    R Wm = half * (l.W + r.W);
    R uxm = half * (l.ux + r.ux);
    R uym = half * (l.uy + r.uy);
    R usq = uxm * uxm + uym * uym;
    R Lam = Wm * Wm - usq;
    R alpha0 = (R)1 + gm1inv * ibln;
    R pm = rm * rcp<R>(bm);
    R rinv = rcp<R>(Lam * Wm);
    R iLam = rinv * Wm;
    R iW = rinv * Lam;
    R UD = rln * Wm;
    R UE = (alpha0 * UD * Wm + pm * usq) * iLam;
    R un = mx * uxm + my * uym;
    R Es = Wm * (alpha0 * rln + pm) * un * iLam;
    R cm = (mt * (UE + pm) + Es) * iW;
    out[0] = rln * (mt * Wm + un);
    out[1] = uxm * cm + pm * mx;
    out[2] = uym * cm + pm * my;
    out[3] = mt * UE + Es;
}

// The two Jiang-Shu WENO5 edge values of one interface from its six stencil
// values V0..V5 (V2, V3 the interface's nodes): vm from V0..V4 (upwind
// left) and vp from V5..V1 (upwind right).  Each is
//   sum_k (d_k/(eps+b_k)^2) q_k / sum_k d_k/(eps+b_k)^2, d = (0.1, 0.6, 0.3),
// written with a single division by multiplying through by the three
// squared denominators.  The candidate values and second differences of the
// two middle candidate stencils, {V1, V2, V3} and {V2, V3, V4}, serve both
// reconstructions (left's 2nd and 3rd candidates are right's 3rd and 2nd)
// and are formed once.
template <typename R>
__device__ __forceinline__ void weno5_lr(R V0, R V1, R V2, R V3, R V4, R V5, R eps, R &vm, R &vp)
{
    const R c13_12 = (R)(13.0 / 12.0), c1_4 = (R)0.25, c1_6 = (R)(1.0 / 6.0);
    const R qa = (-V1 + (R)5 * V2 + (R)2 * V3) * c1_6;
    const R qb = ((R)2 * V2 + (R)5 * V3 - V4) * c1_6;
    const R ta = V1 - (R)2 * V2 + V3, tb = V2 - (R)2 * V3 + V4;
    const R sa = c13_12 * ta * ta, sb = c13_12 * tb * tb;
    {
        R q0 = ((R)2 * V0 - (R)7 * V1 + (R)11 * V2) * c1_6;
        R t0 = V0 - (R)2 * V1 + V2, r0 = V0 - (R)4 * V1 + (R)3 * V2;
        R r1 = V1 - V3, r2 = (R)3 * V2 - (R)4 * V3 + V4;
        R e0 = eps + c13_12 * t0 * t0 + c1_4 * r0 * r0;
        R e1 = eps + sa + c1_4 * r1 * r1;
        R e2 = eps + sb + c1_4 * r2 * r2;
        e0 *= e0; e1 *= e1; e2 *= e2;
        R a0 = (R)0.1 * e1 * e2, a1 = (R)0.6 * e0 * e2, a2 = (R)0.3 * e0 * e1;
        vm = (a0 * q0 + a1 * qa + a2 * qb) * rcp<R>(a0 + a1 + a2);
    }
    {
        R q0 = ((R)2 * V5 - (R)7 * V4 + (R)11 * V3) * c1_6;
        R t0 = V5 - (R)2 * V4 + V3, r0 = V5 - (R)4 * V4 + (R)3 * V3;
        R r1 = V4 - V2, r2 = (R)3 * V3 - (R)4 * V2 + V1;
        R e0 = eps + c13_12 * t0 * t0 + c1_4 * r0 * r0;
        R e1 = eps + sb + c1_4 * r1 * r1;
        R e2 = eps + sa + c1_4 * r2 * r2;
        e0 *= e0; e1 *= e1; e2 *= e2;
        R a0 = (R)0.1 * e1 * e2, a1 = (R)0.6 * e0 * e2, a2 = (R)0.3 * e0 * e1;
        vp = (a0 * q0 + a1 * qb + a2 * qa) * rcp<R>(a0 + a1 + a2);
    }
}

// The two WENO3 edge values of one interface from V0..V3 (V1, V2 its
// nodes): vm from V0, V1, V2 and vp from V3, V2, V1, each
// (a0 q0 + a1 q1)/(a0 + a1) with a_k = d_k/(eps+b_k)^2, d = (1/3, 2/3),
// multiplied through; the candidate on {V1, V2} and its smoothness term
// serve both.
template <typename R>
__device__ __forceinline__ void weno3_lr(R V0, R V1, R V2, R V3, R eps, R &vm, R &vp)
{
    const R q1 = (V1 + V2) * (R)0.5;
    R e1 = eps + (V2 - V1) * (V2 - V1);
    e1 *= e1;
    {
        R q0 = (-V0 + (R)3 * V1) * (R)0.5;
        R e0 = eps + (V1 - V0) * (V1 - V0);
        e0 *= e0;
        R a0 = (R)(1.0 / 3.0) * e1, a1 = (R)(2.0 / 3.0) * e0;
        vm = (a0 * q0 + a1 * q1) * rcp<R>(a0 + a1);
    }
    {
        R q0 = (-V3 + (R)3 * V2) * (R)0.5;
        R e0 = eps + (V2 - V3) * (V2 - V3);
        e0 *= e0;
        R a0 = (R)(1.0 / 3.0) * e1, a1 = (R)(2.0 / 3.0) * e0;
        vp = (a0 * q0 + a1 * q1) * rcp<R>(a0 + a1);
    }
}

__device__ __forceinline__ int sgn_d(double a) { return (a > 0.0) - (a < 0.0); }
__device__ __forceinline__ int sgn_d(float a) { return (a > 0.0f) - (a < 0.0f); }
__device__ __forceinline__ int sgn_d(dual a) { return (a.v > 0.0) - (a.v < 0.0); }
__device__ __forceinline__ bool le(double a, double b) { return a <= b; }
__device__ __forceinline__ bool le(float a, float b) { return a <= b; }
__device__ __forceinline__ bool le(dual a, dual b) { return a.v <= b.v; }

// Scaled eigenvectors of dF_1/dU (Sec. 4) at the rotated state (rho, vn, vt, p)
// with W = 1/sqrt(1 - vn^2 - vt^2): columns dU_m * s_m, s_m = (dU_m . dV_m)^-1/2,
// for the waves (lambda_-, v_n [entropy, d rho = 1], v_n [shear, d v_t = 1],
// lambda_+ [acoustic, dp = 1]).  dU (4 x 4, column per wave) and s are returned
// separately; lam_m, lam_p are the acoustic speeds; gm1i = 1/(Gamma - 1).
template <typename R>
__device__ __forceinline__ void eigen_rhd(R gam, R gm1i, R rho, R vn, R vt, R p, R W,
                                          R dU[4][4], R s[4], R &lam_m, R &lam_p)
{
    R one = (R)1;
    R gg = gam * gm1i;
    R W2 = W * W;
    R iW2 = rcp<R>(W2);                    // 1 - v^2
    R v2 = one - iW2;
    R irp = rcp<R>(rho * p);
    R ip = rho * irp, ir = p * irp;
    R rh = rho + gg * p;                   // rho h
    R c2 = gam * p * rcp<R>(rh);
    R c = sqrt_pos<R>(c2);
    R disc = sqrt_pos<R>(iW2 * (one - v2 * c2 - vn * vn * (one - c2)));
    R den = rcp<R>(one - v2 * c2);
    lam_m = (vn * (one - c2) - c * disc) * den;
    lam_p = (vn * (one - c2) + c * disc) * den;
    R Q = rh * W2;
    R beta = rho * ip;
    R un = W * vn, ut = W * vt;
    R W4 = W2 * W2;
    // entropy wave, d rho = 1:  dU = (W, W^2 v, W^2),  dU.dV = G W/((G-1) rho)
    dU[0][1] = W; dU[1][1] = W2 * vn; dU[2][1] = W2 * vt; dU[3][1] = W2;
    s[1] = rsq<R>(gg * W * ir);
    // shear wave, d v_t = 1:  dU = (rho W^3 vt, 2 rho h W^4 vn vt,
    //   rho h (2 W^4 vt^2 + W^2), 2 rho h W^4 vt),  dU.dV = rho h beta W^3 (1 + W^2 vt^2)
    dU[0][2] = rho * W2 * W * vt;
    dU[1][2] = (R)2 * rh * W4 * vn * vt;
    dU[2][2] = rh * ((R)2 * W4 * vt * vt + W2);
    dU[3][2] = (R)2 * rh * W4 * vt;
    s[2] = rsq<R>(rh * beta * W2 * W * (one + W2 * vt * vt));
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        int m = side == 0 ? 0 : 3;
        R l = side == 0 ? lam_m : lam_p;
        R a = rcp<R>((l - vn) * Q);          // 1 / ((lam - v_n) Q)
        R dvn = (one - vn * l) * a;
        R dvt = -l * vt * a;
        R vdv = vn * dvn + vt * dvt;
        R drho = rho * dvn * a * Q - rho * W2 * vdv;
        // dU/dw dw with dp = 1
        R h1 = drho + gg;                    // d(rho h)
        R dW = W2 * W * vdv;
        dU[0][m] = W * drho + rho * dW;
        dU[1][m] = W2 * vn * h1 + rh * ((R)2 * W4 * vn * vdv + W2 * dvn);
        dU[2][m] = W2 * vt * h1 + rh * ((R)2 * W4 * vt * vdv + W2 * dvt);
        dU[3][m] = W2 * h1 - one + rh * (R)2 * W4 * vdv;
        // dV/dw dw
        R dbeta = drho * ip - beta * ip;
        R dV0 = drho * ir + (drho * ir - ip) * gm1i + dbeta;
        R dV1 = dbeta * un + beta * (W * dvn + vn * dW);
        R dV2 = dbeta * ut + beta * (W * dvt + vt * dW);
        R dV3 = -(dbeta * W + beta * dW);
        s[m] = rsq<R>(dU[0][m] * dV0 + dU[1][m] * dV1 + dU[2][m] * dV2 + dU[3][m] * dV3);
    }
}

}  // namespace esmm
