// bsq_kernels.cu -- sm_103a kernels of one adaptive-AB3 extended Boussinesq
// step (arXiv 1909.04153).  One step is five launches on the domain's stream:
//
//   ctl_ghost   controller (Eqs. 22, 47, 42, 44-46; computed redundantly by
//               every block so no block waits on another) + two ghost layers
//               of w, P, Q (Sec. 3.3) + wave-maker corrections of the line
//               right-hand sides
//   rhs_combine KP07 reconstruction and central-upwind fluxes, bed source,
//               friction, dispersive central differences (Eqs. 11-15), then
//               the AB3 combine (Eqs. 42-43) with compensated accumulation
//   ysolve      y-line tridiagonal solves (Eq. 20) for the Q increment,
//               chunked Thomas with block scans; sponge on Q
//   ghost_q     ghost layers of Q^{n+1} (only for the sequential cross form)
//   xsolve      F* at the new level from Q^{n+1} (Eq. 14), x-line solves
//               (Eq. 19) for the P increment with warp scans, sponge on w and
//               P, and the Eq. 22 rate of the new state (block max + atomic)
//
// Fields are SoA, row-major, x fastest, with a 2-cell halo in y and a 16-byte
// aligned halo in x, so rows can be read as float4 / double2.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "bsq_internal.cuh"
#include "bsq_launch.h"

namespace bsq {

// ------------------------------------------------------------------ helpers

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

__device__ __forceinline__ float trsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double trsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }

// minmod of three arguments; generalized minmod slope (per cell width)
template <typename T>
__device__ __forceinline__ T minmod3(T a, T b, T c)
{
    if (a > (T)0 && b > (T)0 && c > (T)0) return tmin(a, tmin(b, c));
    if (a < (T)0 && b < (T)0 && c < (T)0) return tmax(a, tmax(b, c));
    return (T)0;
}
template <typename T>
__device__ __forceinline__ T gslope(T qm, T q0, T qp, T th)
{
    return minmod3(th * (q0 - qm), (T)0.5 * (qp - qm), th * (qp - q0));
}

// 1 / sqrt(h^4 + max(h^4, eps)) of the desingularised velocity of KP07,
// u = sqrt(2) h m / sqrt(h^4 + max(h^4, eps))
template <typename T>
__device__ __forceinline__ T desing_inv(T h, T eps)
{
    T h2 = h * h;
    T h4 = h2 * h2;
    return trsqrt(h4 + tmax(h4, eps));
}

#define BSQ_SQRT2 1.41421356237309504880

// Linear wave-maker state (eta, P, Q) at (x, y, t), all in FP64.
template <typename T>
__device__ void maker_state(const Dev<T> &D, double x, double y, double t, double &e, double &p, double &q)
{
    double r = D.ramp_time > 0.0 ? tanh(3.0 * t / D.ramp_time) : 1.0;
    double se = 0.0, sp = 0.0, sq = 0.0;
    for (int k = 0; k < D.ncomp; k++) {
        double ek = D.amp[k] * cos(D.kx[k] * x + D.ky[k] * y - D.om[k] * t + D.ph[k]);
        se += ek;
        sp += D.cx[k] * ek;
        sq += D.cy[k] * ek;
    }
    e = r * se;
    p = r * sp;
    q = r * sq;
}

// ------------------------------------------------------------------ controller

// Step size (Eq. 22 with the lazy EMA of Eq. 47, clamps), AB3 weights
// (Eq. 42) and the weights of the F*, G* levels: Eq. 43 with Eqs. 44-46
// collapses to quadratic extrapolation to t_{n+1} minus the value at t_n,
// written here in closed form.  The Euler start (Sec. 3.2.1) covers n < 2.
template <typename T>
__device__ void controller(const Dev<T> &D, double forced_dt, Coef &cf, unsigned &err)
{
    const volatile Ctl *cv = D.ctl;
    long long n = cv->n;
    double t = cv->t, dtm1 = cv->dtm1, dtm2 = cv->dtm2, t_end = cv->t_end;
    long long n_limit = cv->n_limit;
    unsigned cerr = cv->err;
    unsigned long long rb = cv->rate_bits;
    err = 0;
    cf.n = n;
    cf.t0 = t;
    cf.t1 = t;
    cf.dt = 0.0;
    cf.active = 0;
    int s0 = (int)(n % 3);
    cf.s0 = s0;
    cf.s1 = (s0 + 2) % 3;
    cf.s2 = (s0 + 1) % 3;
    cf.wc = (int)(n & 1);
    cf.nlev = n == 0 ? 1 : (n == 1 ? 2 : 3);
    for (int k = 0; k < 3; k++) { cf.beta[k] = 0.0; cf.gam[k] = 0.0; cf.betaf[k] = 0.f; cf.gamf[k] = 0.f; }
    double tol = isfinite(t_end) ? 1e-12 * fmax(1.0, fabs(t_end)) : 0.0;
    if (cerr != 0u || n >= n_limit || !(t < t_end - tol)) return;
    double dt;
    if (forced_dt > 0.0) {
        dt = forced_dt;
    } else {
        double rate = bitsd(rb);
        double dtc;
        if (rate > 0.0) dtc = D.cfl / rate;
        else if (D.dt_max > 0.0) dtc = D.dt_max;
        else { err = ERR_NODT; return; }
        dt = (n == 0 && D.dt_init > 0.0) ? D.dt_init : dtc;
        if (n >= 2 && dt > dtm1) dt = D.ema_alpha * dt + (1.0 - D.ema_alpha) * dtm1;
        if (D.dt_max > 0.0 && dt > D.dt_max) dt = D.dt_max;
        if (dt < D.dt_min) { err = ERR_UNSTABLE; return; }
        double rem = t_end - t;
        if (dt > rem) dt = rem;
    }
    if (!(dt > 0.0)) { err = ERR_NODT; return; }
    if (n == 0) {
        cf.beta[0] = dt;
    } else if (n == 1) {
        cf.beta[0] = dt;
        cf.gam[0] = 1.0;
        cf.gam[1] = -1.0;
    } else {
        double a = dt, b = dtm1, c = dtm2;
        cf.beta[0] = a / 6.0 * (a / b * (2.0 * a + 6.0 * b + 3.0 * c) / (b + c) + 6.0);
        cf.beta[1] = -a / 6.0 * (a / b * (2.0 * a + 3.0 * b + 3.0 * c) / c);
        cf.beta[2] = a / 6.0 * (a / c * (2.0 * a + 3.0 * b) / (b + c));
        // Lagrange weights of t_n, t_{n-1}, t_{n-2} at t_{n+1}, minus e_0
        cf.gam[0] = a * (a + 2.0 * b + c) / (b * (b + c));
        cf.gam[1] = -a * (a + b + c) / (b * c);
        cf.gam[2] = a * (a + b) / (c * (b + c));
    }
    for (int k = 0; k < 3; k++) { cf.betaf[k] = (float)cf.beta[k]; cf.gamf[k] = (float)cf.gam[k]; }
    cf.dt = dt;
    cf.t1 = t + dt;
    cf.active = 1;
}

template <typename T> __device__ __forceinline__ T coefv(const Coef &c, int which, int k);
template <> __device__ __forceinline__ float coefv<float>(const Coef &c, int which, int k)
{
    return which ? c.gamf[k] : c.betaf[k];
}
template <> __device__ __forceinline__ double coefv<double>(const Coef &c, int which, int k)
{
    return which ? c.gam[k] : c.beta[k];
}

// ------------------------------------------------------------------ ghost cells

// Value of ghost cell (i, j) from the current interior: the W/E columns are
// filled first (mirror with P negated, or the maker), then the S/N rows from
// the filled columns (mirror with Q negated, or the maker).
template <typename T>
__device__ void ghost_value(const Dev<T> &D, const T *w, int i, int j, double t, T &gw, T &gP, T &gQ)
{
    int nx = D.nx, ny = D.ny;
    int side = -1;
    bool flipP = false, flipQ = false;
    int si = i, sj = j;
    if (j < 0 || j >= ny) {
        side = j < 0 ? SS : SN;
        if (D.bc[side] != MAKER) {
            sj = j < 0 ? -j - 1 : 2 * ny - 1 - j;
            flipQ = true;
            side = -1;
        }
    }
    if (side < 0 && (si < 0 || si >= nx)) {
        side = si < 0 ? SW : SE;
        if (D.bc[side] != MAKER) {
            si = si < 0 ? -si - 1 : 2 * nx - 1 - si;
            flipP = true;
            side = -1;
        }
    }
    if (side >= 0) {
        double e, p, q;
        maker_state(D, ((double)i + 0.5) * D.dxd, ((double)j + 0.5) * D.dyd, t, e, p, q);
        long long c = fidx(D, i, j);
        T b = D.bC[c];
        T d = tmax(D.w_s - b, (T)0);
        T h = tmax(d + (T)e, (T)0);
        gw = b + h;
        gP = (T)p;
        gQ = (T)q;
        return;
    }
    long long c = fidx(D, si, sj);
    gw = w[c];
    gP = flipP ? -D.P[c] : D.P[c];
    gQ = flipQ ? -D.Q[c] : D.Q[c];
}

// Controller + ghost fill at t_n + maker corrections of the line systems.
template <typename T>
__global__ void __launch_bounds__(256) k_ctl_ghost(Dev<T> D, double forced_dt)
{
    __shared__ Coef scf;
    __shared__ unsigned serr;
    if (threadIdx.x == 0) {
        Coef cf;
        unsigned err;
        controller(D, forced_dt, cf, err);
        scf = cf;
        serr = err;
        if (blockIdx.x == 0) {
            *D.coef = cf;
            if (err) atomicOr(&D.ctl->err, err);
        }
    }
    __syncthreads();
    if (!scf.active) return;
    const double t0 = scf.t0, t1 = scf.t1;
    int nx = D.nx, ny = D.ny;
    T *w = D.w[scf.wc];
    long long nghost = 4LL * ny + 4LL * (nx + 4);
    long long ntot = nghost + 2LL * ny + 2LL * nx;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < ntot;
         idx += (long long)gridDim.x * blockDim.x) {
        if (idx < 4LL * ny) {
            int side = (int)(idx / (2 * ny));
            int rem = (int)(idx % (2 * ny));
            int g = rem / ny + 1, j = rem % ny;
            int i = side == 0 ? -g : nx - 1 + g;
            T a, b, c;
            ghost_value(D, w, i, j, t0, a, b, c);
            long long f = fidx(D, i, j);
            w[f] = a; D.P[f] = b; D.Q[f] = c;
        } else if (idx < nghost) {
            long long k = idx - 4LL * ny;
            int side = (int)(k / (2 * (nx + 4)));
            int rem = (int)(k % (2 * (nx + 4)));
            int g = rem / (nx + 4) + 1, i = rem % (nx + 4) - 2;
            int j = side == 0 ? -g : ny - 1 + g;
            T a, b, c;
            ghost_value(D, w, i, j, t0, a, b, c);
            long long f = fidx(D, i, j);
            w[f] = a; D.P[f] = b; D.Q[f] = c;
        } else {
            long long k = idx - nghost;
            // corrections: -A_0 (g^{n+1} - g^n) of Eq. 19/20 in increment form
            if (k < 2LL * ny) {
                int side = (int)(k / ny), j = (int)(k % ny);
                int s = side == 0 ? SW : SE;
                T corr = (T)0;
                if (D.bc[s] == MAKER) {
                    double x = side == 0 ? -0.5 * D.dxd : ((double)nx + 0.5) * D.dxd;
                    double y = ((double)j + 0.5) * D.dyd;
                    double e0, p0, q0, e1, p1, q1;
                    maker_state(D, x, y, t0, e0, p0, q0);
                    maker_state(D, x, y, t1, e1, p1, q1);
                    double a = side == 0 ? D.cW[j] : D.cE[j];
                    corr = (T)(-a * (p1 - p0));
                }
                (side == 0 ? D.corrW : D.corrE)[j] = corr;
            } else {
                k -= 2LL * ny;
                int side = (int)(k / nx), i = (int)(k % nx);
                int s = side == 0 ? SS : SN;
                T corr = (T)0;
                if (D.bc[s] == MAKER) {
                    double x = ((double)i + 0.5) * D.dxd;
                    double y = side == 0 ? -0.5 * D.dyd : ((double)ny + 0.5) * D.dyd;
                    double e0, p0, q0, e1, p1, q1;
                    maker_state(D, x, y, t0, e0, p0, q0);
                    maker_state(D, x, y, t1, e1, p1, q1);
                    double a = side == 0 ? D.cS[i] : D.cN[i];
                    corr = (T)(-a * (q1 - q0));
                }
                (side == 0 ? D.corrS : D.corrN)[i] = corr;
            }
        }
    }
}

// Ghost layers of Q at t_{n+1} (after the y-line solves), for F*(Q^{n+1}).
template <typename T>
__global__ void __launch_bounds__(256) k_ghost_q(Dev<T> D)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    int nx = D.nx, ny = D.ny;
    long long nghost = 4LL * ny + 4LL * (nx + 4);
    T *w = D.w[cf.wc ^ 1];
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nghost;
         idx += (long long)gridDim.x * blockDim.x) {
        int i, j;
        if (idx < 4LL * ny) {
            int side = (int)(idx / (2 * ny));
            int rem = (int)(idx % (2 * ny));
            int g = rem / ny + 1;
            j = rem % ny;
            i = side == 0 ? -g : nx - 1 + g;
        } else {
            long long k = idx - 4LL * ny;
            int side = (int)(k / (2 * (nx + 4)));
            int rem = (int)(k % (2 * (nx + 4)));
            int g = rem / (nx + 4) + 1;
            i = rem % (nx + 4) - 2;
            j = side == 0 ? -g : ny - 1 + g;
        }
        T a, b, c;
        ghost_value(D, w, i, j, cf.t1, a, b, c);
        D.Q[fidx(D, i, j)] = c;
    }
}

// ------------------------------------------------------------------ RHS + combine

template <typename T>
__device__ __forceinline__ void reconstruct(T wm, T w0, T wp, T Pm, T P0, T Pp, T Qm, T Q0, T Qp,
                                            T blo, T bhi, T th, T &wl, T &wh, T &Pl, T &Ph,
                                            T &Ql, T &Qh)
{
    T sw = gslope(wm, w0, wp, th);
    T sP = gslope(Pm, P0, Pp, th);
    T sQ = gslope(Qm, Q0, Qp, th);
    T a = w0 + (T)0.5 * sw, b = w0 - (T)0.5 * sw;
    if (a < bhi) { a = bhi; b = (T)2 * w0 - bhi; }
    else if (b < blo) { b = blo; a = (T)2 * w0 - blo; }
    wl = b; wh = a;
    Pl = P0 - (T)0.5 * sP; Ph = P0 + (T)0.5 * sP;
    Ql = Q0 - (T)0.5 * sQ; Qh = Q0 + (T)0.5 * sQ;
}

// Central-upwind flux across one face; DIR 0: x-face, 1: y-face.
template <typename T, int DIR>
__device__ __forceinline__ void cu_flux(T bf, T wL, T PL, T QL, T wR, T PR, T QR, T g, T eps,
                                        T &H0, T &H1, T &H2)
{
    T hL = tmax(wL - bf, (T)0), hR = tmax(wR - bf, (T)0);
    T iL = (T)BSQ_SQRT2 * hL * desing_inv(hL, eps);
    T iR = (T)BSQ_SQRT2 * hR * desing_inv(hR, eps);
    T uL = iL * PL, vL = iL * QL, uR = iR * PR, vR = iR * QR;
    T pL = hL * uL, qL = hL * vL, pR = hR * uR, qR = hR * vR;
    T cL = tsqrt(g * hL), cR = tsqrt(g * hR);
    T unL = DIR == 0 ? uL : vL, unR = DIR == 0 ? uR : vR;
    T ap = tmax(tmax(unL + cL, unR + cR), (T)0);
    T am = tmin(tmin(unL - cL, unR - cR), (T)0);
    T den = ap - am;
    if (!(den > (T)0)) { H0 = H1 = H2 = (T)0; return; }
    T inv = (T)1 / den;
    T FL0, FL1, FL2, FR0, FR1, FR2;
    if (DIR == 0) {
        FL0 = pL; FL1 = pL * uL + (T)0.5 * g * hL * hL; FL2 = qL * uL;
        FR0 = pR; FR1 = pR * uR + (T)0.5 * g * hR * hR; FR2 = qR * uR;
    } else {
        FL0 = qL; FL1 = pL * vL; FL2 = qL * vL + (T)0.5 * g * hL * hL;
        FR0 = qR; FR1 = pR * vR; FR2 = qR * vR + (T)0.5 * g * hR * hR;
    }
    T k = ap * am * inv;
    H0 = (ap * FL0 - am * FR0) * inv + k * (hR - hL);
    H1 = (ap * FL1 - am * FR1) * inv + k * (pR - pL);
    H2 = (ap * FL2 - am * FR2) * inv + k * (qR - qL);
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) k_rhs_combine(Dev<T> D)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    constexpr int SX = TX + 4, SY = TY + 4;
    __shared__ T sw[SY][SX], sP[SY][SX], sQ[SY][SX], sEta[SY][SX], sD[SY][SX], sB[SY][SX];
    __shared__ T sK[SY + 1][SX + 1];
    __shared__ T sHx[3][TY][TX + 1];
    __shared__ T sHy[3][TY + 1][TX];

    const int tid = threadIdx.y * TX + threadIdx.x;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int nx = D.nx, ny = D.ny;
    const T *w = D.w[cf.wc];

    // 1. stage w, P, Q (2-cell halo) and the bed corners
    for (int q = tid; q < SX * SY; q += TX * TY) {
        int a = q % SX, b = q / SX;
        int i = min(i0 + a - 2, nx + 1), j = min(j0 + b - 2, ny + 1);
        long long c = fidx(D, i, j);
        sw[b][a] = w[c];
        sP[b][a] = D.P[c];
        sQ[b][a] = D.Q[c];
    }
    for (int q = tid; q < (SX + 1) * (SY + 1); q += TX * TY) {
        int a = q % (SX + 1), b = q / (SX + 1);
        int i = min(i0 + a - 2, nx + 2), j = min(j0 + b - 2, ny + 2);
        sK[b][a] = D.corner[(long long)(j + 2) * D.cpitch + (i + 2)];
    }
    __syncthreads();
    // 2. cell-centre bed (mean of the 4 face values), still depth, eta = h - d
    for (int q = tid; q < SX * SY; q += TX * TY) {
        int a = q % SX, b = q / SX;
        T bw = (T)0.5 * (sK[b][a] + sK[b + 1][a]);
        T be = (T)0.5 * (sK[b][a + 1] + sK[b + 1][a + 1]);
        T bs = (T)0.5 * (sK[b][a] + sK[b][a + 1]);
        T bn = (T)0.5 * (sK[b + 1][a] + sK[b + 1][a + 1]);
        T bc = (T)0.25 * (bw + be + bs + bn);
        T d = tmax(D.w_s - bc, (T)0);
        sB[b][a] = bc;
        sD[b][a] = d;
        sEta[b][a] = tmax(sw[b][a] - bc, (T)0) - d;
    }
    __syncthreads();
    // 3. face fluxes: x-faces (TX+1) x TY, then y-faces TX x (TY+1)
    const T th = D.theta, g = D.g, eps = D.eps;
    for (int q = tid; q < (TX + 1) * TY + TX * (TY + 1); q += TX * TY) {
        if (q < (TX + 1) * TY) {
            int fa = q % (TX + 1), r = q / (TX + 1);
            int b = r + 2, aL = fa + 1, aR = fa + 2;
            T bf = (T)0.5 * (sK[b][aR] + sK[b + 1][aR]);
            T bLw = (T)0.5 * (sK[b][aL] + sK[b + 1][aL]);
            T bRe = (T)0.5 * (sK[b][aR + 1] + sK[b + 1][aR + 1]);
            T wl, wh, Pl, Ph, Ql, Qh, wl2, wh2, Pl2, Ph2, Ql2, Qh2;
            reconstruct(sw[b][aL - 1], sw[b][aL], sw[b][aL + 1], sP[b][aL - 1], sP[b][aL], sP[b][aL + 1],
                        sQ[b][aL - 1], sQ[b][aL], sQ[b][aL + 1], bLw, bf, th, wl, wh, Pl, Ph, Ql, Qh);
            reconstruct(sw[b][aR - 1], sw[b][aR], sw[b][aR + 1], sP[b][aR - 1], sP[b][aR], sP[b][aR + 1],
                        sQ[b][aR - 1], sQ[b][aR], sQ[b][aR + 1], bf, bRe, th, wl2, wh2, Pl2, Ph2, Ql2, Qh2);
            T H0, H1, H2;
            cu_flux<T, 0>(bf, wh, Ph, Qh, wl2, Pl2, Ql2, g, eps, H0, H1, H2);
            sHx[0][r][fa] = H0; sHx[1][r][fa] = H1; sHx[2][r][fa] = H2;
        } else {
            int q2 = q - (TX + 1) * TY;
            int c = q2 % TX, fb = q2 / TX;
            int a = c + 2, bL = fb + 1, bU = fb + 2;
            T bf = (T)0.5 * (sK[bU][a] + sK[bU][a + 1]);
            T bLs = (T)0.5 * (sK[bL][a] + sK[bL][a + 1]);
            T bUn = (T)0.5 * (sK[bU + 1][a] + sK[bU + 1][a + 1]);
            T wl, wh, Pl, Ph, Ql, Qh, wl2, wh2, Pl2, Ph2, Ql2, Qh2;
            reconstruct(sw[bL - 1][a], sw[bL][a], sw[bL + 1][a], sP[bL - 1][a], sP[bL][a], sP[bL + 1][a],
                        sQ[bL - 1][a], sQ[bL][a], sQ[bL + 1][a], bLs, bf, th, wl, wh, Pl, Ph, Ql, Qh);
            reconstruct(sw[bU - 1][a], sw[bU][a], sw[bU + 1][a], sP[bU - 1][a], sP[bU][a], sP[bU + 1][a],
                        sQ[bU - 1][a], sQ[bU][a], sQ[bU + 1][a], bf, bUn, th, wl2, wh2, Pl2, Ph2, Ql2, Qh2);
            T H0, H1, H2;
            cu_flux<T, 1>(bf, wh, Ph, Qh, wl2, Pl2, Ql2, g, eps, H0, H1, H2);
            sHy[0][fb][c] = H0; sHy[1][fb][c] = H1; sHy[2][fb][c] = H2;
        }
    }
    __syncthreads();

    // 4. per interior cell: E, F, G, F*, G* and the AB3 combine
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = i0 + tx, j = j0 + ty;
    bool clamped = false;
    if (i < nx && j < ny) {
        const int a = tx + 2, b = ty + 2;
        const T rdx = D.rdx, rdy = D.rdy;
        T divx0 = (sHx[0][ty][tx + 1] - sHx[0][ty][tx]) * rdx;
        T divx1 = (sHx[1][ty][tx + 1] - sHx[1][ty][tx]) * rdx;
        T divx2 = (sHx[2][ty][tx + 1] - sHx[2][ty][tx]) * rdx;
        T divy0 = (sHy[0][ty + 1][tx] - sHy[0][ty][tx]) * rdy;
        T divy1 = (sHy[1][ty + 1][tx] - sHy[1][ty][tx]) * rdy;
        T divy2 = (sHy[2][ty + 1][tx] - sHy[2][ty][tx]) * rdy;
        T bW = (T)0.5 * (sK[b][a] + sK[b + 1][a]);
        T bE = (T)0.5 * (sK[b][a + 1] + sK[b + 1][a + 1]);
        T bS = (T)0.5 * (sK[b][a] + sK[b][a + 1]);
        T bN = (T)0.5 * (sK[b + 1][a] + sK[b + 1][a + 1]);
        T w0 = sw[b][a], P0 = sP[b][a], Q0 = sQ[b][a], bc = sB[b][a];
        T srcx = -g * (bE - bW) * rdx * (w0 - (T)0.5 * (bE + bW));
        T srcy = -g * (bN - bS) * rdy * (w0 - (T)0.5 * (bN + bS));
        T fr1 = (T)0, fr2 = (T)0;
        if (D.friction != (T)0) {
            T h = tmax(w0 - bc, (T)0);
            T iv = (T)BSQ_SQRT2 * h * desing_inv(h, eps);
            T u = iv * P0, v = iv * Q0;
            T sp = tsqrt(u * u + v * v);
            fr1 = D.friction * u * sp;
            fr2 = D.friction * v * sp;
        }
        // dispersive central differences (Eqs. 12-15)
        const T d = sD[b][a];
        const T half_rdx = (T)0.5 * rdx, half_rdy = (T)0.5 * rdy;
        const T ddx = (sD[b][a + 1] - sD[b][a - 1]) * half_rdx;
        const T ddy = (sD[b + 1][a] - sD[b - 1][a]) * half_rdy;
        const T rdx2 = rdx * rdx, rdy2 = rdy * rdy;
        T e_xx = (sEta[b][a + 1] - (T)2 * sEta[b][a] + sEta[b][a - 1]) * rdx2;
        T e_yy = (sEta[b + 1][a] - (T)2 * sEta[b][a] + sEta[b - 1][a]) * rdy2;
        T e_xy = (sEta[b + 1][a + 1] - sEta[b - 1][a + 1] - sEta[b + 1][a - 1] + sEta[b - 1][a - 1]) *
                 ((T)0.25 * rdx * rdy);
        T e_xxx = (sEta[b][a + 2] - (T)2 * sEta[b][a + 1] + (T)2 * sEta[b][a - 1] - sEta[b][a - 2]) *
                  ((T)0.5 * rdx2 * rdx);
        T e_yyy = (sEta[b + 2][a] - (T)2 * sEta[b + 1][a] + (T)2 * sEta[b - 1][a] - sEta[b - 2][a]) *
                  ((T)0.5 * rdy2 * rdy);
        T eyy_p = (sEta[b + 1][a + 1] - (T)2 * sEta[b][a + 1] + sEta[b - 1][a + 1]) * rdy2;
        T eyy_m = (sEta[b + 1][a - 1] - (T)2 * sEta[b][a - 1] + sEta[b - 1][a - 1]) * rdy2;
        T exx_p = (sEta[b + 1][a + 1] - (T)2 * sEta[b + 1][a] + sEta[b + 1][a - 1]) * rdx2;
        T exx_m = (sEta[b - 1][a + 1] - (T)2 * sEta[b - 1][a] + sEta[b - 1][a - 1]) * rdx2;
        T e_xyy = (eyy_p - eyy_m) * half_rdx;
        T e_xxy = (exx_p - exx_m) * half_rdy;
        const T Bg = D.Bd * g;
        T dispx = Bg * d * d * d * (e_xxx + e_xyy) + Bg * d * d * (ddx * ((T)2 * e_xx + e_yy) + ddy * e_xy);
        T dispy = Bg * d * d * d * (e_yyy + e_xxy) + Bg * d * d * (ddy * ((T)2 * e_yy + e_xx) + ddx * e_xy);
        T E = -divx0 - divy0;
        T F = -divx1 - divy1 + srcx - fr1 + dispx;
        T G = -divx2 - divy2 + srcy - fr2 + dispy;
        const T kB = D.Bd + (T)1 / (T)3;
        const T sixth = (T)1 / (T)6;
        T Q_x = (sQ[b][a + 1] - sQ[b][a - 1]) * half_rdx;
        T Q_y = (sQ[b + 1][a] - sQ[b - 1][a]) * half_rdy;
        T Q_xy = (sQ[b + 1][a + 1] - sQ[b - 1][a + 1] - sQ[b + 1][a - 1] + sQ[b - 1][a - 1]) *
                 ((T)0.25 * rdx * rdy);
        T P_x = (sP[b][a + 1] - sP[b][a - 1]) * half_rdx;
        T P_y = (sP[b + 1][a] - sP[b - 1][a]) * half_rdy;
        T P_xy = (sP[b + 1][a + 1] - sP[b - 1][a + 1] - sP[b + 1][a - 1] + sP[b - 1][a - 1]) *
                 ((T)0.25 * rdx * rdy);
        T Fs = d * ddx * Q_y * sixth + d * ddy * Q_x * sixth + kB * d * d * Q_xy;
        T Gs = d * ddy * P_x * sixth + d * ddx * P_y * sixth + kB * d * d * P_xy;

        // AB3 / Euler combine (Eqs. 42-43)
        const long long c = fidx(D, i, j);
        const long long fs = D.fstride;
        T *H = D.hist;
        const T b0 = coefv<T>(cf, 0, 0), b1 = coefv<T>(cf, 0, 1), b2 = coefv<T>(cf, 0, 2);
        const T g0 = coefv<T>(cf, 1, 0), g1 = coefv<T>(cf, 1, 1), g2 = coefv<T>(cf, 1, 2);
        T dw = b0 * E, dU = b0 * F, dV = b0 * G + g0 * Gs;
        const bool extrap = D.cross_mode == 0;
        if (extrap) dU += g0 * Fs;
        if (cf.nlev >= 2) {
            const long long o = (long long)cf.s1 * fs + c;
            dw += b1 * H[0 * 3 * fs + o];
            dU += b1 * H[1 * 3 * fs + o];
            dV += b1 * H[2 * 3 * fs + o] + g1 * H[4 * 3 * fs + o];
            if (extrap) dU += g1 * H[3 * 3 * fs + o];
        }
        if (cf.nlev >= 3) {
            const long long o = (long long)cf.s2 * fs + c;
            dw += b2 * H[0 * 3 * fs + o];
            dU += b2 * H[1 * 3 * fs + o];
            dV += b2 * H[2 * 3 * fs + o] + g2 * H[4 * 3 * fs + o];
            if (extrap) dU += g2 * H[3 * 3 * fs + o];
        }
        if (!extrap) dU -= Fs;  // F*(Q^{n+1}) is added by the x-line kernel
        {
            const long long o = (long long)cf.s0 * fs + c;
            H[0 * 3 * fs + o] = E;
            H[1 * 3 * fs + o] = F;
            H[2 * 3 * fs + o] = G;
            if (extrap) H[3 * 3 * fs + o] = Fs;
            H[4 * 3 * fs + o] = Gs;
        }
        // w^{n+1} = w^n + dw with compensated accumulation, then h >= 0
        T wn, cwn = (T)0;
        if (D.kahan) {
            T cw = D.cw[c];
            T y = dw - cw;
            wn = w0 + y;
            cwn = (wn - w0) - y;
        } else {
            wn = w0 + dw;
        }
        if (wn < bc) { wn = bc; cwn = (T)0; clamped = true; }
        D.w[cf.wc ^ 1][c] = wn;
        if (D.kahan) D.cw[c] = cwn;
        D.dU[c] = dU;
        D.dV[c] = dV;
    }
    int nclamp = __syncthreads_count(clamped);
    if (tid == 0 && nclamp) atomicAdd(&D.ctl->clamps, (unsigned long long)nclamp);
    if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0) {
        // commit the step in the controller state (the controller kernel of
        // this step has finished; no block of this kernel reads Ctl)
        Ctl *ct = D.ctl;
        ct->dtm2 = ct->dtm1;
        ct->dtm1 = cf.dt;
        ct->last_dt = cf.dt;
        ct->t = cf.t1;
        ct->n = cf.n + 1;
        ct->rate_bits = 0ull;
    }
}

// ------------------------------------------------------------------ y-line solves

// Thread (column c, chunk k) owns rows [k*KCH, (k+1)*KCH) of one column.
// Forward elimination y_j = m_j r_j + e_j y_{j-1} and back substitution
// x_j = y_j - c'_j x_{j+1} are affine recurrences: each thread composes its
// chunk, a block scan over the chunks of a column supplies the value entering
// each chunk, and the chunk is finished from registers.
template <typename T, int KCH>
__global__ void k_ysolve(Dev<T> D, int CW, int NCH)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    extern __shared__ unsigned char smem_raw[];
    T *sA = reinterpret_cast<T *>(smem_raw);
    T *sB = sA + CW * NCH;
    const int t = threadIdx.x;
    const int c = t % CW, k = t / CW;
    const int i = blockIdx.x * CW + c;
    const int nx = D.nx, ny = D.ny;
    const bool col = i < nx;
    const int j0 = k * KCH;
    T r[KCH], m[KCH], e[KCH];
    T A = (T)1, B = (T)0;
#pragma unroll
    for (int q = 0; q < KCH; q++) {
        int j = j0 + q;
        bool v = col && j < ny;
        long long o = v ? fidx(D, i, j) : 0;
        T rr = v ? D.dV[o] : (T)0;
        if (v && j == 0) rr += D.corrS[i];
        if (v && j == ny - 1) rr += D.corrN[i];
        T mm = v ? D.fym[o] : (T)0;
        T ee = v ? D.fye[o] : (T)1;
        r[q] = rr; m[q] = mm; e[q] = ee;
        B = mm * rr + ee * B;
        A = ee * A;
    }
    // inclusive scan over the chunks of the column (earlier chunks first)
    sA[t] = A; sB[t] = B;
    for (int s = 1; s < NCH; s <<= 1) {
        __syncthreads();
        T Ap = (T)1, Bp = (T)0;
        bool has = k >= s;
        if (has) { Ap = sA[t - s * CW]; Bp = sB[t - s * CW]; }
        __syncthreads();
        if (has) { B = A * Bp + B; A = A * Ap; }
        sA[t] = A; sB[t] = B;
    }
    __syncthreads();
    T y = k > 0 ? sB[t - CW] : (T)0;
    __syncthreads();
    T cp[KCH];
    T al = (T)0, be = (T)1;
#pragma unroll
    for (int q = 0; q < KCH; q++) {
        int j = j0 + q;
        bool v = col && j < ny;
        y = m[q] * r[q] + e[q] * y;
        r[q] = y;  // r now holds y
        T cc = v ? D.fyc[fidx(D, i, v ? j : 0)] : (T)0;
        cp[q] = cc;
        al = al + be * y;
        be = -cc * be;
    }
    // inclusive scan from the last chunk backwards: X_k = al_k + be_k X_{k+1}
    sA[t] = al; sB[t] = be;
    for (int s = 1; s < NCH; s <<= 1) {
        __syncthreads();
        T ap = (T)0, bp = (T)1;
        bool has = k + s < NCH;
        if (has) { ap = sA[t + s * CW]; bp = sB[t + s * CW]; }
        __syncthreads();
        if (has) { al = al + be * ap; be = be * bp; }
        sA[t] = al; sB[t] = be;
    }
    __syncthreads();
    T x = k + 1 < NCH ? sA[t + CW] : (T)0;
    if (!col) return;
#pragma unroll
    for (int q = KCH - 1; q >= 0; q--) {
        int j = j0 + q;
        if (j < ny) {
            x = r[q] - cp[q] * x;
            long long o = fidx(D, i, j);
            T Qo = D.Q[o], Qn, cn = (T)0;
            if (D.kahan) {
                T cq = D.cQ[o];
                T yy = x - cq;
                Qn = Qo + yy;
                cn = (Qn - Qo) - yy;
            } else {
                Qn = Qo + x;
            }
            T gm = D.gx[i] * D.gy[j];
            if (gm < (T)1) { Qn *= gm; cn *= gm; }
            D.Q[o] = Qn;
            if (D.kahan) D.cQ[o] = cn;
        }
    }
}

// ------------------------------------------------------------------ x-line solves

template <typename T> struct VecT;
template <> struct VecT<float> { typedef float4 type; static constexpr int N = 4; };
template <> struct VecT<double> { typedef double2 type; static constexpr int N = 2; };

template <typename T>
__device__ __forceinline__ void vload(const T *p, T *out)
{
    typedef typename VecT<T>::type V;
    V v = *reinterpret_cast<const V *>(p);
    const T *s = reinterpret_cast<const T *>(&v);
#pragma unroll
    for (int q = 0; q < VecT<T>::N; q++) out[q] = s[q];
}
template <typename T>
__device__ __forceinline__ void vstore(T *p, const T *in)
{
    typedef typename VecT<T>::type V;
    V v;
    T *s = reinterpret_cast<T *>(&v);
#pragma unroll
    for (int q = 0; q < VecT<T>::N; q++) s[q] = in[q];
    *reinterpret_cast<V *>(p) = v;
}

// Row segment of VEC elements per lane plus one neighbour on each side.
template <typename T, int VEC>
__device__ __forceinline__ void load_halo_row(const T *row, int ibase, int lane, T *v)
{
    vload(row + ibase, v + 1);
    T left = __shfl_up_sync(0xffffffffu, v[VEC], 1);
    T right = __shfl_down_sync(0xffffffffu, v[1], 1);
    if (lane == 0) left = row[ibase - 1];
    if (lane == 31) right = row[ibase + VEC];
    v[0] = left;
    v[VEC + 1] = right;
}

template <typename T>
__global__ void k_xsolve(Dev<T> D, int nseg)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    constexpr int VEC = VecT<T>::N;
    constexpr int SEG = 32 * VEC;
    extern __shared__ unsigned char smem_raw[];
    T *ybuf = reinterpret_cast<T *>(smem_raw) + (size_t)threadIdx.y * nseg * SEG;
    __shared__ double wmax[32];
    const int lane = threadIdx.x;
    const int j = blockIdx.x * blockDim.y + threadIdx.y;
    const int nx = D.nx, ny = D.ny;
    const bool rowok = j < ny;
    const int jr = rowok ? j : ny - 1;  // keep loads in bounds for idle rows
    const long long rowo = fidx(D, 0, jr);
    const T *dUr = D.dU + rowo, *mr = D.fxm + rowo, *er = D.fxe + rowo, *cr = D.fxc + rowo;
    const bool seq = D.cross_mode != 0;
    const T half_rdx = (T)0.5 * D.rdx, half_rdy = (T)0.5 * D.rdy, q_rdxy = (T)0.25 * D.rdx * D.rdy;
    const T kB = D.Bd + (T)1 / (T)3, sixth = (T)1 / (T)6;
    const T corrW = D.corrW[jr], corrE = D.corrE[jr];

    // forward elimination, segment by segment, carry = y at the last element
    T carry = (T)0;
    for (int s = 0; s < nseg; s++) {
        const int ib = s * SEG + lane * VEC;
        T r[VEC], m[VEC], e[VEC];
        vload(dUr + ib, r);
        vload(mr + ib, m);
        vload(er + ib, e);
        if (seq) {
            // F* of Eq. 14 at the new level from Q^{n+1} (ghosts at t_{n+1})
            T q0[VEC + 2], qm[VEC + 2], qp[VEC + 2], b0[VEC + 2], bm[VEC + 2], bp[VEC + 2];
            load_halo_row<T, VEC>(D.Q + rowo, ib, lane, q0);
            load_halo_row<T, VEC>(D.Q + rowo - D.pitch, ib, lane, qm);
            load_halo_row<T, VEC>(D.Q + rowo + D.pitch, ib, lane, qp);
            load_halo_row<T, VEC>(D.bC + rowo, ib, lane, b0);
            load_halo_row<T, VEC>(D.bC + rowo - D.pitch, ib, lane, bm);
            load_halo_row<T, VEC>(D.bC + rowo + D.pitch, ib, lane, bp);
#pragma unroll
            for (int q = 0; q < VEC; q++) {
                T d = tmax(D.w_s - b0[q + 1], (T)0);
                T ddx = (tmax(D.w_s - b0[q + 2], (T)0) - tmax(D.w_s - b0[q], (T)0)) * half_rdx;
                T ddy = (tmax(D.w_s - bp[q + 1], (T)0) - tmax(D.w_s - bm[q + 1], (T)0)) * half_rdy;
                T Q_x = (q0[q + 2] - q0[q]) * half_rdx;
                T Q_y = (qp[q + 1] - qm[q + 1]) * half_rdy;
                T Q_xy = (qp[q + 2] - qm[q + 2] - qp[q] + qm[q]) * q_rdxy;
                r[q] += d * ddx * Q_y * sixth + d * ddy * Q_x * sixth + kB * d * d * Q_xy;
            }
        }
#pragma unroll
        for (int q = 0; q < VEC; q++) {
            int i = ib + q;
            if (i == 0) r[q] += corrW;
            if (i == nx - 1) r[q] += corrE;
            if (i >= nx) { r[q] = (T)0; m[q] = (T)0; e[q] = (T)1; }
        }
        T A = (T)1, B = (T)0;
#pragma unroll
        for (int q = 0; q < VEC; q++) { B = m[q] * r[q] + e[q] * B; A = e[q] * A; }
        // inclusive warp scan, lower lanes first
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T Ap = __shfl_up_sync(0xffffffffu, A, o);
            T Bp = __shfl_up_sync(0xffffffffu, B, o);
            if (lane >= o) { B = A * Bp + B; A = A * Ap; }
        }
        T Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
        if (lane == 0) { Ae = (T)1; Be = (T)0; }
        T y = Ae * carry + Be;
#pragma unroll
        for (int q = 0; q < VEC; q++) { y = m[q] * r[q] + e[q] * y; r[q] = y; }
        vstore(ybuf + ib, r);
        carry = __shfl_sync(0xffffffffu, y, 31);
    }
    __syncwarp();

    // back substitution from the last segment, carry = x at the first element
    T xcarry = (T)0;
    T rate = (T)0;
    bool bad = false;
    T *Pr = D.P + rowo, *cPr = D.cP + rowo;
    T *wr = D.w[cf.wc ^ 1] + rowo, *cwr = D.cw + rowo;
    const T *Qr = D.Q + rowo, *bCr = D.bC + rowo;
    const T gyj = D.gy[jr];
    for (int s = nseg - 1; s >= 0; s--) {
        const int ib = s * SEG + lane * VEC;
        T y[VEC], cc[VEC];
        vload(ybuf + ib, y);
        vload(cr + ib, cc);
#pragma unroll
        for (int q = 0; q < VEC; q++)
            if (ib + q >= nx) { y[q] = (T)0; cc[q] = (T)0; }
        // lane map: x_first = al + be * x_after
        T al = (T)0, be = (T)1;
#pragma unroll
        for (int q = VEC - 1; q >= 0; q--) { al = y[q] - cc[q] * al; be = -cc[q] * be; }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T ap = __shfl_down_sync(0xffffffffu, al, o);
            T bp = __shfl_down_sync(0xffffffffu, be, o);
            if (lane + o < 32) { al = al + be * ap; be = be * bp; }
        }
        T an = __shfl_down_sync(0xffffffffu, al, 1), bn = __shfl_down_sync(0xffffffffu, be, 1);
        if (lane == 31) { an = (T)0; bn = (T)1; }
        T x = an + bn * xcarry;
        T xs[VEC];
#pragma unroll
        for (int q = VEC - 1; q >= 0; q--) { x = y[q] - cc[q] * x; xs[q] = x; }
        xcarry = __shfl_sync(0xffffffffu, xs[0], 0);

        // P^{n+1} = P^n + x (compensated), sponge on w and P, Eq. 22 rate
        if (rowok) {
            T Pv[VEC], cPv[VEC], wv[VEC], Qv[VEC], bv[VEC];
            vload(Pr + ib, Pv);
            if (D.kahan) vload(cPr + ib, cPv);
            vload(wr + ib, wv);
            vload(Qr + ib, Qv);
            vload(bCr + ib, bv);
#pragma unroll
            for (int q = 0; q < VEC; q++) {
                const int i = ib + q;
                if (i >= nx) continue;
                T Pn, cn = (T)0;
                if (D.kahan) {
                    T yy = xs[q] - cPv[q];
                    Pn = Pv[q] + yy;
                    cn = (Pn - Pv[q]) - yy;
                } else {
                    Pn = Pv[q] + xs[q];
                }
                T wq = wv[q];
                T gm = D.gx[i] * gyj;
                if (gm < (T)1) {
                    T h = tmax(wq - bv[q], (T)0), d = tmax(D.w_s - bv[q], (T)0);
                    wq = bv[q] + (d + gm * (h - d));
                    wr[i] = wq;
                    if (D.kahan) cwr[i] = (T)0;
                    Pn *= gm;
                    cn *= gm;
                }
                Pv[q] = Pn;
                cPv[q] = cn;
                T h = tmax(wq - bv[q], (T)0);
                T iv = (T)BSQ_SQRT2 * h * desing_inv(h, D.eps);
                T u = iv * Pn, v = iv * Qv[q];
                T cc2 = tsqrt(D.g * h);
                T rq = tmax((fabs(u) + cc2) * D.rdx, (fabs(v) + cc2) * D.rdy);
                rate = tmax(rate, rq);
                if (!isfinite(wq) || !isfinite(Pn) || !isfinite(Qv[q])) bad = true;
            }
            vstore(Pr + ib, Pv);
            if (D.kahan) vstore(cPr + ib, cPv);
        }
    }
    // block max of the rate, one atomic per block
    double rr = (double)rate;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rr = fmax(rr, __shfl_xor_sync(0xffffffffu, rr, o));
    bool anybad = __any_sync(0xffffffffu, bad);
    if (lane == 0) wmax[threadIdx.y] = anybad ? -1.0 : rr;
    __syncthreads();
    if (threadIdx.y == 0 && lane == 0) {
        double mx = 0.0;
        bool fl = false;
        for (int q = 0; q < (int)blockDim.y; q++) {
            if (wmax[q] < 0.0) fl = true;
            else mx = fmax(mx, wmax[q]);
        }
        if (fl) atomicOr(&D.ctl->err, ERR_NONFINITE);
        atomicMax(&D.ctl->rate_bits, dbits(mx));
    }
}

// ------------------------------------------------------------------ utilities

// Eq. 22 rate of the current state (used at creation and after a restore).
template <typename T>
__global__ void __launch_bounds__(256) k_rate(Dev<T> D, int wc)
{
    __shared__ double red[8];
    double mx = 0.0;
    const T *w = D.w[wc];
    long long ncell = (long long)D.nx * D.ny;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < ncell;
         q += (long long)gridDim.x * blockDim.x) {
        int i = (int)(q % D.nx), j = (int)(q / D.nx);
        long long c = fidx(D, i, j);
        T h = tmax(w[c] - D.bC[c], (T)0);
        T iv = (T)BSQ_SQRT2 * h * desing_inv(h, D.eps);
        T u = iv * D.P[c], v = iv * D.Q[c];
        T cc = tsqrt(D.g * h);
        T r = tmax((fabs(u) + cc) * D.rdx, (fabs(v) + cc) * D.rdy);
        mx = fmax(mx, (double)r);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); q++) mx = fmax(mx, red[q]);
        atomicMax(&D.ctl->rate_bits, dbits(mx));
    }
}

// Interior field into a compact nx*ny array of T.
template <typename T>
__global__ void __launch_bounds__(256) k_extract(Dev<T> D, int wc, int field, T *out)
{
    long long ncell = (long long)D.nx * D.ny;
    const T *w = D.w[wc];
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < ncell;
         q += (long long)gridDim.x * blockDim.x) {
        int i = (int)(q % D.nx), j = (int)(q / D.nx);
        long long c = fidx(D, i, j);
        T b = D.bC[c];
        T h = tmax(w[c] - b, (T)0);
        T v;
        switch (field) {
        case 0: v = h - tmax(D.w_s - b, (T)0); break;
        case 1: v = D.P[c]; break;
        case 2: v = D.Q[c]; break;
        case 3: v = h; break;
        default: v = w[c]; break;
        }
        out[q] = v;
    }
}

// Per-block partial sums of h (for the mass diagnostic).
template <typename T>
__global__ void __launch_bounds__(256) k_mass(Dev<T> D, int wc, double *partial)
{
    __shared__ double red[8];
    double s = 0.0;
    const T *w = D.w[wc];
    long long ncell = (long long)D.nx * D.ny;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < ncell;
         q += (long long)gridDim.x * blockDim.x) {
        int i = (int)(q % D.nx), j = (int)(q / D.nx);
        long long c = fidx(D, i, j);
        s += (double)tmax(w[c] - D.bC[c], (T)0);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); q++) s += red[q];
        partial[blockIdx.x] = s;
    }
}

__global__ void k_set_limits(Ctl *ctl, double t_end, long long max_steps)
{
    ctl->t_end = t_end;
    ctl->n_limit = max_steps > 0 ? ctl->n + max_steps : 0x7fffffffffffffffLL;
}

// ------------------------------------------------------------------ launchers

template <typename T>
static void ysolve_shape(int nx, int ny, int &CW, int &NCH, int &kch)
{
    kch = sizeof(T) == 4 ? 32 : 16;
    NCH = (ny + kch - 1) / kch;
    CW = 32;
    while (CW > 1 && CW * NCH > 512) CW >>= 1;
    (void)nx;
}

template <typename T>
int step_shape_ok(int nx, int ny)
{
    int CW, NCH, kch;
    ysolve_shape<T>(nx, ny, CW, NCH, kch);
    return CW * NCH <= 1024;
}

template <typename T>
static int xsolve_rows(int nseg)
{
    size_t per = (size_t)nseg * 32 * VecT<T>::N * sizeof(T);
    int rows = 4;
    while (rows > 1 && rows * per > 96 * 1024) rows >>= 1;
    return rows;
}

template <typename T>
size_t xsolve_smem(int nx)
{
    constexpr int SEG = 32 * VecT<T>::N;
    int nseg = (nx + SEG - 1) / SEG;
    return (size_t)xsolve_rows<T>(nseg) * nseg * SEG * sizeof(T);
}

template <typename T>
int row_segment() { return 32 * VecT<T>::N; }

template <typename T>
cudaError_t configure(int nx)
{
    cudaError_t e = cudaFuncSetAttribute(k_xsolve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)xsolve_smem<T>(nx) + 1024);
    return e;
}

// One step: five launches on stream st.  With ev != nullptr, events ev[0..5]
// are recorded before each launch and after the last (kernel timing).
template <typename T>
static cudaError_t step_impl(const Dev<T> &D, cudaStream_t st, double forced_dt, cudaEvent_t *ev)
{
    const int nx = D.nx, ny = D.ny;
    long long nwork = 4LL * ny + 4LL * (nx + 4) + 2LL * ny + 2LL * nx;
    int gb = (int)((nwork + 255) / 256);
    if (ev) cudaEventRecord(ev[0], st);
    k_ctl_ghost<T><<<gb, 256, 0, st>>>(D, forced_dt);
    if (ev) cudaEventRecord(ev[1], st);
    constexpr int TX = 32, TY = 8;
    dim3 g1((nx + TX - 1) / TX, (ny + TY - 1) / TY);
    k_rhs_combine<T, TX, TY><<<g1, dim3(TX, TY), 0, st>>>(D);
    if (ev) cudaEventRecord(ev[2], st);
    int CW, NCH, kch;
    ysolve_shape<T>(nx, ny, CW, NCH, kch);
    size_t sm = 2 * (size_t)CW * NCH * sizeof(T);
    if (kch == 32)
        k_ysolve<T, 32><<<(nx + CW - 1) / CW, CW * NCH, sm, st>>>(D, CW, NCH);
    else
        k_ysolve<T, 16><<<(nx + CW - 1) / CW, CW * NCH, sm, st>>>(D, CW, NCH);
    if (ev) cudaEventRecord(ev[3], st);
    if (D.cross_mode != 0) {
        long long ng = 4LL * ny + 4LL * (nx + 4);
        k_ghost_q<T><<<(int)((ng + 255) / 256), 256, 0, st>>>(D);
    }
    if (ev) cudaEventRecord(ev[4], st);
    constexpr int SEG = 32 * VecT<T>::N;
    int nseg = (nx + SEG - 1) / SEG;
    int rows = xsolve_rows<T>(nseg);
    size_t smx = (size_t)rows * nseg * SEG * sizeof(T);
    k_xsolve<T><<<(ny + rows - 1) / rows, dim3(32, rows), smx, st>>>(D, nseg);
    if (ev) cudaEventRecord(ev[5], st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step(const Dev<T> &D, cudaStream_t st, double forced_dt)
{
    return step_impl<T>(D, st, forced_dt, nullptr);
}

template <typename T>
cudaError_t launch_step_timed(const Dev<T> &D, cudaStream_t st, double forced_dt, cudaEvent_t *ev)
{
    return step_impl<T>(D, st, forced_dt, ev);
}

template <typename T>
cudaError_t launch_rate(const Dev<T> &D, cudaStream_t st, int wc)
{
    long long ncell = (long long)D.nx * D.ny;
    int gb = (int)std::min<long long>((ncell + 255) / 256, 1024);
    k_rate<T><<<gb, 256, 0, st>>>(D, wc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extract(const Dev<T> &D, cudaStream_t st, int wc, int field, T *out)
{
    long long ncell = (long long)D.nx * D.ny;
    int gb = (int)std::min<long long>((ncell + 255) / 256, 4096);
    k_extract<T><<<gb, 256, 0, st>>>(D, wc, field, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mass(const Dev<T> &D, cudaStream_t st, int wc, double *partial, int nblocks)
{
    k_mass<T><<<nblocks, 256, 0, st>>>(D, wc, partial);
    return cudaGetLastError();
}

cudaError_t launch_set_limits(Ctl *ctl, cudaStream_t st, double t_end, long long max_steps)
{
    k_set_limits<<<1, 1, 0, st>>>(ctl, t_end, max_steps);
    return cudaGetLastError();
}

#define BSQ_INST(T)                                                                              \
    template int step_shape_ok<T>(int, int);                                                     \
    template size_t xsolve_smem<T>(int);                                                         \
    template int row_segment<T>();                                                               \
    template cudaError_t configure<T>(int);                                                      \
    template cudaError_t launch_step<T>(const Dev<T> &, cudaStream_t, double);                   \
    template cudaError_t launch_step_timed<T>(const Dev<T> &, cudaStream_t, double, cudaEvent_t *);\
    template cudaError_t launch_rate<T>(const Dev<T> &, cudaStream_t, int);                      \
    template cudaError_t launch_extract<T>(const Dev<T> &, cudaStream_t, int, int, T *);         \
    template cudaError_t launch_mass<T>(const Dev<T> &, cudaStream_t, int, double *, int);
BSQ_INST(float)
BSQ_INST(double)

}  // namespace bsq
