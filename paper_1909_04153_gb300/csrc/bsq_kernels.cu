// bsq_kernels.cu -- sm_103a kernels of one adaptive-AB3 extended Boussinesq
// step (arXiv 1909.04153).  In the default single-precision configuration a
// step is five launches on the domain's stream:
//
//   ghost       two ghost layers of w, P, Q at t_n (Sec. 3.3) and the
//               wave-maker corrections of the line right-hand sides
//   rhs_combine KP07 reconstruction and central-upwind fluxes, bed source,
//               dispersive central differences (Eqs. 11-15), the AB3 combine
//               (Eqs. 42-43) with compensated accumulation, and the chunk
//               summaries of the y-line solves
//   yscan       scans of the y-line chunk summaries, per column
//   yapply      y-line substitutions (Eq. 20) for the Q increment; sponge on Q
//   xsolve      F* at the new level from Q^{n+1} (Eq. 14), x-line solves
//               (Eq. 19) for the P increment with warp scans, sponge on w and
//               P, the Eq. 22 rate of the new state, and in its last block the
//               controller of the next step (Eqs. 22, 47, 42, 44-46)
//
// Other kernel shapes (tiled or one-column-per-lane RHS, block-scan
// y-solver, TMA-staged x-solvers) are selected by bsq_params.tune and
// parity-tested.
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

// Selections between doubles on the integer pipe.  GB300 runs FP64 at 1/64
// of the FP32 rate and a compare or a min/max of doubles takes an FP64 issue
// slot like an add.  The bits of a double read as a signed integer, with the
// magnitude bits of negative values flipped and -0 taken as +0, order the
// values exactly as the FP64 compare does (NaNs aside: a non-finite state is
// flagged anyway), so these pick the same double without the FP64 pipe.
__device__ __forceinline__ long long dkey(double x)
{
    long long i = __double_as_longlong(x);
    i = i == (long long)0x8000000000000000ULL ? 0LL : i;
    return i ^ ((i >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double tmax(double a, double b) { return dkey(a) > dkey(b) ? a : b; }
__device__ __forceinline__ double tmin(double a, double b) { return dkey(a) < dkey(b) ? a : b; }
template <typename T>
__device__ __forceinline__ bool tlt(T a, T b) { return a < b; }
__device__ __forceinline__ bool tlt(double a, double b) { return dkey(a) < dkey(b); }
template <typename T>
__device__ __forceinline__ bool tfinite(T x) { return isfinite(x); }
__device__ __forceinline__ bool tfinite(double x) { return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff; }
// minmod of two slopes: the one nearer zero when both have the same sign and
// neither is zero, else 0.  In double precision from the bits: for two
// positive doubles the smaller integer is the smaller value, for two negative
// ones the smaller integer is the one nearer zero.
template <typename T>
__device__ __forceinline__ T minmod2(T a, T c)
{
    const T mn = tmin(a, c), mx = tmax(a, c);
    return mn > (T)0 ? mn : (mx < (T)0 ? mx : (T)0);
}
__device__ __forceinline__ double minmod2(double a, double c)
{
    const long long ia = __double_as_longlong(a), ic = __double_as_longlong(c);
    const bool keep = ((ia ^ ic) >= 0) && ((ia << 1) != 0) && ((ic << 1) != 0);
    return keep ? __longlong_as_double(ia < ic ? ia : ic) : 0.0;
}

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
    T a = q0 - qm, c = qp - q0;
    if (th == (T)1) {
        // theta = 1: the centred difference (a + c)/2 lies between a and c, so
        // the minmod of the three equals the minmod of a and c (bitwise)
        // (branch-free: both positive -> the smaller, both negative -> the
        // larger, otherwise 0)
        return minmod2(a, c);
    }
    return minmod3(th * a, (T)0.5 * (qp - qm), th * c);
}

// 1 / sqrt(h^4 + max(h^4, eps)) of the desingularised velocity of KP07,
// u = sqrt(2) h m / sqrt(h^4 + max(h^4, eps))
#define BSQ_SQRT2 1.41421356237309504880

template <typename T>
__device__ __forceinline__ T desing_inv(T h, T eps)
{
    T h2 = h * h;
    T h4 = h2 * h2;
    return trsqrt(h4 + tmax(h4, eps));
}

// Desingularised velocity factor and celerity of a depth h (KP07, Sec. 3.4):
// iv = sqrt(2) h / sqrt(h^4 + max(h^4, eps)), so u = iv P, v = iv Q, and
// c = sqrt(g h).  Single precision evaluates them as written.  Double
// precision, whose square roots and divisions are long instruction sequences
// at GB300's FP64 rate, takes both from one reciprocal square root r of h
// where h^4 >= eps: there iv = 1/h exactly, so iv = r^2 and c = sqrt(g) h r;
// the near-dry side (h^4 < eps) keeps the formula.  The rounded h^4 grows
// with h, so h^4 < eps holds exactly below one double, hdry (found once on
// the host); the test compares h with it, and h^4 is formed only near dry.
template <typename T>
struct IvC {
    T iv, c;
};
__device__ __forceinline__ IvC<float> ivc(float h, float g, float sqrtg, float eps, float hdry)
{
    (void)sqrtg;
    (void)hdry;
    return {(float)BSQ_SQRT2 * h * desing_inv(h, eps), sqrtf(g * h)};
}
__device__ __forceinline__ IvC<double> ivc(double h, double g, double sqrtg, double eps, double hdry)
{
    (void)g;
    const double r = rsqrt(tmax(h, 1e-300));
    IvC<double> o;
    o.c = sqrtg * h * r;
    o.iv = r * r;
    // h >= +0 (or NaN, which fails the test as it fails h^4 < eps)
    if (__double_as_longlong(h) < __double_as_longlong(hdry)) {
        const double h2 = h * h, h4 = h2 * h2;
        o.iv = BSQ_SQRT2 * h * rsqrt(h4 + eps);
    }
    return o;
}


// vector loads and stores of K contiguous elements (float4 / double2)
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
template <typename T, int K>
__device__ __forceinline__ void vload_k(const T *p, T *out)
{
#pragma unroll
    for (int v = 0; v < K; v += VecT<T>::N) vload(p + v, out + v);
}
template <typename T, int K>
__device__ __forceinline__ void vstore_k(T *p, const T *in)
{
#pragma unroll
    for (int v = 0; v < K; v += VecT<T>::N) vstore(p + v, in + v);
}

// K contiguous elements of a row starting at ib, plus one neighbour on each
// side (v[0] and v[K+1]); neighbours come from the adjacent lanes, and from
// memory at the ends of a warp.
template <typename T, int K>
__device__ __forceinline__ void load_halo_chunk(const T *row, int ib, int lane, T *v)
{
    vload_k<T, K>(row + ib, v + 1);
    T left = __shfl_up_sync(0xffffffffu, v[K], 1);
    T right = __shfl_down_sync(0xffffffffu, v[1], 1);
    if (lane == 0) left = row[ib - 1];
    if (lane == 31) right = row[ib + K];
    v[0] = left;
    v[K + 1] = right;
}

// Per-column stride of the y-line chunk summaries: the chunk count rounded up
// to 8, so a lane's 8 chunks are one aligned vector
__host__ __device__ __forceinline__ int ychunk_stride(int nch) { return (nch + 7) & ~7; }

// KP07 bed at a cell centre from its corners k00 = (i, j), k10 = (i+1, j),
// k01 = (i, j+1), k11 = (i+1, j+1): the mean of the four face values, each
// face the mean of its two corners, rounded step by step in this order
__device__ __forceinline__ float bed_centre(float k00, float k10, float k01, float k11)
{
    const float bw = __fmul_rn(0.5f, __fadd_rn(k00, k01)), be = __fmul_rn(0.5f, __fadd_rn(k10, k11));
    const float bs = __fmul_rn(0.5f, __fadd_rn(k00, k10)), bn = __fmul_rn(0.5f, __fadd_rn(k01, k11));
    return __fmul_rn(0.25f, __fadd_rn(__fadd_rn(__fadd_rn(bw, be), bs), bn));
}
__device__ __forceinline__ double bed_centre(double k00, double k10, double k01, double k11)
{
    return 0.25 * (0.5 * (k00 + k01) + 0.5 * (k10 + k11) + 0.5 * (k00 + k10) + 0.5 * (k01 + k11));
}

// Wave-maker ramp r(t) = tanh(3 t / ramp_time) (1 without a ramp).
template <typename T>
__device__ double maker_ramp(const Dev<T> &D, double t)
{
    return D.ramp_time > 0.0 ? tanh(3.0 * t / D.ramp_time) : 1.0;
}

// sin and cos of a phase given in FP64, to single precision, for the
// single-precision path: the phase is reduced by quadrants in FP64,
// r = ph - n pi/2 with |r| <= pi/4, then the Taylor series of sin (through
// r^9) and cos (through r^10) are summed in FP32 (truncation below 2e-9 on
// |r| <= pi/4) and rotated back by the quadrant n mod 4.
__device__ __forceinline__ void sincos_phase_f(double ph, float &s, float &c)
{
    const double n = rint(ph * 0.63661977236758134);  // 2 / pi
    const float r = (float)(ph - n * 1.5707963267948966);
    const float r2 = r * r;
    const float sr = r * (1.0f - r2 * (1.0f / 6.0f - r2 * (1.0f / 120.0f - r2 * (1.0f / 5040.0f - r2 * (1.0f / 362880.0f)))));
    const float cr = 1.0f - r2 * (0.5f - r2 * (1.0f / 24.0f - r2 * (1.0f / 720.0f - r2 * (1.0f / 40320.0f - r2 * (1.0f / 3628800.0f)))));
    const int q = (int)((long long)n & 3);
    s = q == 0 ? sr : (q == 1 ? cr : (q == 2 ? -sr : -cr));
    c = q == 0 ? cr : (q == 1 ? -sr : (q == 2 ? -cr : sr));
}

// Linear wave-maker state (eta, P, Q) at (x, y, t) with ramp value r, in FP64
// (the double-precision path).
template <typename T>
__device__ void maker_state(const Dev<T> &D, double x, double y, double t, double r, double &e, double &p, double &q)
{
    double se = 0.0, sp = 0.0, sq = 0.0;
    for (int k = 0; k < D.ncomp; k++) {
        const double ph = D.kx[k] * x + D.ky[k] * y - D.om[k] * t + D.ph[k];
        const double ek = D.amp[k] * cos(ph);
        se += ek;
        sp += D.cx[k] * ek;
        sq += D.cy[k] * ek;
    }
    e = r * se;
    p = r * sp;
    q = r * sq;
}

// Increments of the maker fluxes from (t0, r0) to (t1, r1) at (x, y), and Q
// at t1, in FP64.  They enter the boundary rows of the line systems as
// -A (g^{n+1} - g^n).
template <typename T>
__device__ void maker_increment(const Dev<T> &D, double x, double y, double t0, double t1, double r0, double r1,
                                double &dp, double &dq, double &q1)
{
    double e0, p0, q0, e1, p1;
    maker_state(D, x, y, t0, r0, e0, p0, q0);
    maker_state(D, x, y, t1, r1, e1, p1, q1);
    dp = p1 - p0;
    dq = q1 - q0;
}

// ---- the single-precision maker
//
// A component's phase kx x + ky y + phi - omega t splits into a spatial part,
// fixed at every point where the maker is evaluated, and a temporal part
// shared by all points.  The spatial part's cos and sin are tabulated once at
// set-up (FP64, rounded to FP32; k_setup_mtab), the temporal part's once per
// step and block in shared memory (maker_step), and a point's value is the
// rotation  cos(s + t) = cos s cos t - sin s sin t  in FP32: no FP64
// arithmetic per point and component.
//
// Maker points: the two ghost layers (g = 1, 2) of each side, each over the
// side's length plus two cells past either end, W from 0, E from 2 (ny + 4),
// S from 4 (ny + 4), N from 4 (ny + 4) + 2 (nx + 4); the boundary points of
// the line systems are the cells of layer 1.  Table layout [component][point].
template <typename T>
__device__ __forceinline__ int maker_point(const Dev<T> &D, int side, int i, int j)
{
    const int ly = D.ny + 4, lx = D.nx + 4;
    if (side == SW) return (-i - 1) * ly + j + 2;
    if (side == SE) return 2 * ly + (i - D.nx) * ly + j + 2;
    if (side == SS) return 4 * ly + (-j - 1) * lx + i + 2;
    return 4 * ly + 2 * lx + (j - D.ny) * lx + i + 2;
}

// Per-component factors of one step: cos and sin of -omega t, sin d and
// cos d - 1 of d = -omega (t_next - t), and a, a cx, a cy; two float4 per
// component, f[2k] = (cos, sin, sin d, cos d - 1) and f[2k + 1] =
// (a, a cx, a cy, 0).  For |d| <= 1/4 (a step below a 25th of the period, the
// usual case) sin d and cos d - 1 come from their Taylor series, truncated
// below 1e-8 relative; larger steps take sin d and -2 sin^2(d/2) in FP64.
struct MakerStep {
    const float4 *f;
};

// Shared-memory bytes of maker_step for a domain with nc components.
__host__ __device__ constexpr int maker_step_bytes(int nc) { return 2 * nc * (int)sizeof(float4); }

// Fills the factors for the calling block (all its threads take part; one
// __syncthreads).  Dynamic shared memory of maker_step_bytes(ncomp).
template <typename T>
__device__ MakerStep maker_step(const Dev<T> &D, double t, double t_next)
{
    extern __shared__ float4 maker_sm[];
    for (int k = threadIdx.x; k < D.ncomp; k += blockDim.x) {
        float s, c;
        sincos_phase_f(-D.om[k] * t, s, c);
        const double dd = -D.om[k] * (t_next - t);
        float sd, cm1;
        if (fabs(dd) <= 0.25) {
            const float d = (float)dd, d2 = d * d;
            sd = d * (1.0f - d2 * (1.0f / 6.0f - d2 * (1.0f / 120.0f)));
            cm1 = -d2 * (0.5f - d2 * (1.0f / 24.0f - d2 * (1.0f / 720.0f)));
        } else {
            const double sh = sin(0.5 * dd);
            sd = (float)sin(dd);
            cm1 = (float)(-2.0 * sh * sh);
        }
        const float ak = (float)D.amp[k];
        maker_sm[2 * k] = make_float4(c, s, sd, cm1);
        maker_sm[2 * k + 1] = make_float4(ak, (float)D.cx[k] * ak, (float)D.cy[k] * ak, 0.0f);
    }
    __syncthreads();
    return MakerStep{maker_sm};
}

// The table is read in batches of MB components, all loads of a batch issued
// before their use: a point's sum is a chain of load latencies, one per batch
// (a handful of points per block, so little else hides them).  32 for the
// single-domain ghost kernels (a few dozen blocks), 16 for the batched one,
// whose thousand-odd blocks want the registers for residency.  The loads
// carry an L2 evict-last policy, so the table (a few megabytes, read every step)
// tends to stay in L2 while the step's streaming kernels pass through.
constexpr int MK_BATCH_ONE = 32, MK_BATCH_MANY = 16;
// Makers of at most MK_FEW components take a kernel compiled with batches of
// that size: the launch is a chain of latencies, and a fraction of the code
// (fewer unrolled loads to fetch cold, fewer registers) shortens it.
constexpr int MK_FEW = 4;

__device__ __forceinline__ unsigned long long l2_keep_policy()
{
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ float2 ld_keep(const float2 *p, unsigned long long pol)
{
    float2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}

// Maker state (eta, P, Q) at maker point pt and the factors' time, ramp r.
template <int MB>
__device__ __forceinline__ void maker_state_tab(const Dev<float> &D, const MakerStep &m, int pt, float r, float &e,
                                                float &p, float &q)
{
    float se = 0.0f, sp = 0.0f, sq = 0.0f;
    const float2 *tb = D.mtab + pt;
    const int nc = D.ncomp;
    const unsigned long long pol = l2_keep_policy();
    for (int k0 = 0; k0 < nc; k0 += MB) {
        float2 cs[MB];
#pragma unroll
        for (int u = 0; u < MB; u++)
            cs[u] = k0 + u < nc ? ld_keep(tb + (size_t)(k0 + u) * D.mpts, pol) : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int u = 0; u < MB; u++) {
            if (k0 + u < nc) {
                const float4 f = m.f[2 * (k0 + u)], g = m.f[2 * (k0 + u) + 1];
                const float c = cs[u].x * f.x - cs[u].y * f.y;
                se += g.x * c;
                sp += g.y * c;
                sq += g.z * c;
            }
        }
    }
    e = r * se;
    p = r * sp;
    q = r * sq;
}

// Increments of the maker fluxes at maker point pt from (t, r0) to
// (t_next, r1), and Q at t_next.  The increment is a small difference of
// two maker values; it is formed from the identity
//   r1 cos(ph0 + d) - r0 cos(ph0) = cos(ph0) ((r1 - r0) + r1 (cos d - 1)) - r1 sin(ph0) sin d
// so that it keeps single-precision relative accuracy instead of the
// absolute error of two cosines.
template <int MB>
__device__ __forceinline__ void maker_increment_tab(const Dev<float> &D, const MakerStep &m, int pt, float dr,
                                                    float r1, float &dp, float &dq, float &q1)
{
    float sp = 0.0f, sq = 0.0f, sq1 = 0.0f;
    const float2 *tb = D.mtab + pt;
    const int nc = D.ncomp;
    const unsigned long long pol = l2_keep_policy();
    for (int k0 = 0; k0 < nc; k0 += MB) {
        float2 cs[MB];
#pragma unroll
        for (int u = 0; u < MB; u++)
            cs[u] = k0 + u < nc ? ld_keep(tb + (size_t)(k0 + u) * D.mpts, pol) : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int u = 0; u < MB; u++) {
            if (k0 + u < nc) {
                const float4 f = m.f[2 * (k0 + u)], g = m.f[2 * (k0 + u) + 1];
                const float c0 = cs[u].x * f.x - cs[u].y * f.y;
                const float s0 = cs[u].y * f.x + cs[u].x * f.y;
                const float term = c0 * (dr + r1 * f.w) - r1 * s0 * f.z;
                const float c1 = c0 + (c0 * f.w - s0 * f.z);
                sp += g.y * term;
                sq += g.z * term;
                sq1 += g.z * c1;
            }
        }
    }
    dp = sp;
    dq = sq;
    q1 = r1 * sq1;
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
    } else if (D.cfl <= 0.0) {
        // fixed step (Eqs. 16-18), landing on t_end
        dt = D.dt_init;
        double rem = t_end - t;
        if (dt > rem) dt = rem;
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
    cf.ramp0 = maker_ramp(D, cf.t0);
    cf.ramp1 = maker_ramp(D, cf.t1);
    cf.active = 1;
}

// Controller for the step about to start (one thread); forced_dt > 0 replays a step size.
template <typename T>
__global__ void k_prologue(Dev<T> D, double forced_dt, double t_end, long long max_steps)
{
    // limits of the run, then the controller of its first step
    D.ctl->t_end = t_end;
    D.ctl->n_limit = max_steps > 0 ? D.ctl->n + max_steps : 0x7fffffffffffffffLL;
    Coef cf;
    unsigned err;
    controller(D, forced_dt, cf, err);
    *D.coef = cf;
    if (err) atomicOr(&D.ctl->err, err);
    D.ctl->done_count = 0u;
}

// End of a step, in the last x-solver block to finish (thread 0 only, after
// this block's atomicMax of the rate): the Eq. 22 rate of the new state is then
// complete, so the controller of the next step runs here.
template <typename T>
__device__ void next_step_controller(const Dev<T> &D, double forced_dt_next, unsigned nparts)
{
    __threadfence();
    const unsigned ticket = atomicAdd(&D.ctl->done_count, 1u);
    if (ticket == nparts - 1) {
        __threadfence();
        Coef cf;
        unsigned err;
        controller(D, forced_dt_next, cf, err);
        *D.coef = cf;
        if (err) atomicOr(&D.ctl->err, err);
        D.ctl->done_count = 0u;
    }
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
// The single-precision path evaluates the maker from the table with the
// step factors m (filled for time t); the double-precision path directly.
template <typename T, int MB>
__device__ void ghost_value(const Dev<T> &D, const MakerStep &m, const T *w, int i, int j, double t, double ramp,
                            T &gw, T &gP, T &gQ)
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
        // a maker cell; a corner cell next to a mirrored S/N side is the mirror
        // (Q negated) of the maker column cell (i, sj) it faces
        T e, p, q;
        if constexpr (sizeof(T) == 4) {
            maker_state_tab<MB>(D, m, maker_point(D, side, i, sj), (float)ramp, e, p, q);
        } else {
            maker_state(D, ((double)i + 0.5) * D.dxd, ((double)sj + 0.5) * D.dyd, t, ramp, e, p, q);
        }
        long long c = fidx(D, i, sj);
        T b = D.bC[c];
        T d = tmax(D.w_s - b, (T)0);
        T h = tmax(d + e, (T)0);
        gw = b + h;
        gP = p;
        gQ = flipQ ? -q : q;
        return;
    }
    long long c = fidx(D, si, sj);
    gw = w[c];
    gP = flipP ? -D.P[c] : D.P[c];
    gQ = flipQ ? -D.Q[c] : D.Q[c];
}

// Ghost fill at t_n + maker corrections of the line systems (the controller of
// this step ran at the end of the previous step, or in the prologue).
template <typename T, int MB>
__device__ __forceinline__ void ghost_body(const Dev<T> &D, long long first, long long stride)
{
    const Coef scf = *D.coef;
    if (!scf.active) return;
    const double t0 = scf.t0, t1 = scf.t1, r0 = scf.ramp0, r1 = scf.ramp1;
    MakerStep m{};
    if constexpr (sizeof(T) == 4) {
        if (D.ncomp > 0) m = maker_step(D, t0, t1);  // block-uniform
    }
    int nx = D.nx, ny = D.ny;
    T *w = D.w[scf.wc];
    // 32-bit index arithmetic: the perimeter work is far below 2^31 items
    const int nghost = 4 * ny + 4 * (nx + 4);
    const int ntot = nghost + 2 * ny + 2 * nx;
    for (int idx = (int)first; idx < ntot; idx += (int)stride) {
        if (idx < 4 * ny) {
            int side = idx / (2 * ny);
            int rem = idx - side * 2 * ny;
            int g = rem / ny + 1, j = rem - (g - 1) * ny;
            int i = side == 0 ? -g : nx - 1 + g;
            T a, b, c;
            ghost_value<T, MB>(D, m, w, i, j, t0, r0, a, b, c);
            long long f = fidx(D, i, j);
            w[f] = a; D.P[f] = b; D.Q[f] = c;
        } else if (idx < nghost) {
            int k = idx - 4 * ny;
            int side = k / (2 * (nx + 4));
            int rem = k - side * 2 * (nx + 4);
            int g = rem / (nx + 4) + 1, i = rem - (g - 1) * (nx + 4) - 2;
            int j = side == 0 ? -g : ny - 1 + g;
            T a, b, c;
            ghost_value<T, MB>(D, m, w, i, j, t0, r0, a, b, c);
            long long f = fidx(D, i, j);
            w[f] = a; D.P[f] = b; D.Q[f] = c;
        } else {
            int k = idx - nghost;
            // corrections: -A_0 (g^{n+1} - g^n) of Eq. 19/20 in increment form
            if (k < 2 * ny) {
                int side = k / ny, j = k - side * ny;
                int s = side == 0 ? SW : SE;
                T corr = (T)0;
                if (D.bc[s] == MAKER) {
                    double dp, dq, q1;
                    if constexpr (sizeof(T) == 4) {
                        float fp, fq, fq1;
                        maker_increment_tab<MB>(D, m, maker_point(D, s, side == 0 ? -1 : nx, j), (float)(r1 - r0),
                                            (float)r1, fp, fq, fq1);
                        dp = fp; dq = fq; q1 = fq1;
                    } else {
                        double x = side == 0 ? -0.5 * D.dxd : ((double)nx + 0.5) * D.dxd;
                        double y = ((double)j + 0.5) * D.dyd;
                        maker_increment(D, x, y, t0, t1, r0, r1, dp, dq, q1);
                    }
                    double a = side == 0 ? D.cW[j] : D.cE[j];
                    corr = (T)(-a * dp);
                    (side == 0 ? D.mqW : D.mqE)[j] = (T)q1;
                }
                (side == 0 ? D.corrW : D.corrE)[j] = corr;
            } else {
                k -= 2 * ny;
                int side = k / nx, i = k - side * nx;
                int s = side == 0 ? SS : SN;
                T corr = (T)0;
                if (D.bc[s] == MAKER) {
                    const int jg = side == 0 ? -1 : ny;
                    double x = ((double)i + 0.5) * D.dxd;
                    double y = ((double)jg + 0.5) * D.dyd;
                    double dp, dq, q1;
                    if constexpr (sizeof(T) == 4) {
                        float fp, fq, fq1;
                        maker_increment_tab<MB>(D, m, maker_point(D, s, i, jg), (float)(r1 - r0), (float)r1, fp, fq, fq1);
                        dp = fp; dq = fq; q1 = fq1;
                    } else {
                        maker_increment(D, x, y, t0, t1, r0, r1, dp, dq, q1);
                    }
                    double a = side == 0 ? D.cS[i] : D.cN[i];
                    corr = (T)(-a * dq);
                    (side == 0 ? D.mqS : D.mqN)[i + 1] = (T)q1;
                    if (i == 0 || i == nx - 1) {
                        // the corner columns -1 and nx of the ghost row
                        const int ic = i == 0 ? -1 : nx;
                        if constexpr (sizeof(T) == 4) {
                            float fp, fq, fq1;
                            maker_increment_tab<MB>(D, m, maker_point(D, s, ic, jg), (float)(r1 - r0), (float)r1, fp, fq,
                                                fq1);
                            q1 = fq1;
                        } else {
                            double e1, p1;
                            maker_state(D, ((double)ic + 0.5) * D.dxd, y, t1, r1, e1, p1, q1);
                        }
                        (side == 0 ? D.mqS : D.mqN)[ic + 1] = (T)q1;
                    }
                }
                (side == 0 ? D.corrS : D.corrN)[i] = corr;
            }
        }
    }
}

template <typename T, int MB = MK_BATCH_ONE>
__global__ void __launch_bounds__(256) k_ghost(Dev<T> D)
{
    ghost_body<T, MB>(D, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// Ghost layers of Q at t_{n+1} (after the y-line solves), for F*(Q^{n+1}).
template <typename T>
__global__ void __launch_bounds__(256) k_ghost_q(Dev<T> D)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    MakerStep m{};
    if constexpr (sizeof(T) == 4) {
        if (D.ncomp > 0) m = maker_step(D, cf.t1, cf.t1);  // block-uniform
    }
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
        ghost_value<T, MK_BATCH_ONE>(D, m, w, i, j, cf.t1, cf.ramp1, a, b, c);
        D.Q[fidx(D, i, j)] = c;
    }
}

// ------------------------------------------------------------------ RHS + combine

template <typename T>
__device__ __forceinline__ void reconstruct_tail(T w0, T sw, T P0, T sP, T Q0, T sQ, T blo, T bhi,
                                                 T &wl, T &wh, T &Pl, T &Ph, T &Ql, T &Qh);
template <typename T>
__device__ __forceinline__ void reconstruct(T wm, T w0, T wp, T Pm, T P0, T Pp, T Qm, T Q0, T Qp,
                                            T blo, T bhi, T th, T &wl, T &wh, T &Pl, T &Ph,
                                            T &Ql, T &Qh)
{
    reconstruct_tail(w0, gslope(wm, w0, wp, th), P0, gslope(Pm, P0, Pp, th), Q0, gslope(Qm, Q0, Qp, th),
                     blo, bhi, wl, wh, Pl, Ph, Ql, Qh);
}
// theta = 1 from the one-sided differences a = q0 - qm and c = qp - q0, which
// a caller that walks the cells can pass on from one cell to the next
template <typename T>
__device__ __forceinline__ void reconstruct_d(T w0, T aw, T cw, T P0, T aP, T cP, T Q0, T aQ, T cQ,
                                              T blo, T bhi, T &wl, T &wh, T &Pl, T &Ph, T &Ql, T &Qh)
{
    reconstruct_tail(w0, minmod2(aw, cw), P0, minmod2(aP, cP), Q0, minmod2(aQ, cQ), blo, bhi, wl, wh, Pl, Ph, Ql,
                     Qh);
}
template <typename T>
__device__ __forceinline__ void reconstruct_tail(T w0, T sw, T P0, T sP, T Q0, T sQ, T blo, T bhi,
                                                 T &wl, T &wh, T &Pl, T &Ph, T &Ql, T &Qh)
{
    T a = w0 + (T)0.5 * sw, b = w0 - (T)0.5 * sw;
    // positivity: a face value below the face bed is raised to it and the
    // other face value mirrored about w0 (selects, no branches)
    const bool hi_low = tlt(a, bhi), lo_low = !hi_low && tlt(b, blo);
    wh = hi_low ? bhi : (lo_low ? (T)2 * w0 - blo : a);
    wl = hi_low ? (T)2 * w0 - bhi : (lo_low ? blo : b);
    Pl = P0 - (T)0.5 * sP; Ph = P0 + (T)0.5 * sP;
    Ql = Q0 - (T)0.5 * sQ; Qh = Q0 + (T)0.5 * sQ;
}

// ------------------------------------------------------------------ RHS + combine, sliding window

// Face state of KP07 on one side of a face: depth and desingularised velocities
// and celerity; the discharges are recomputed as h u, h v.
template <typename T>
struct FaceSt {
    T h, u, v, c;
};

__device__ __forceinline__ float trcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double trcp(double x) { return 1.0 / x; }

template <typename T>
__device__ __forceinline__ FaceSt<T> face_state(T wf, T Pf, T Qf, T bf, T g, T sqrtg, T eps, T hdry)
{
    FaceSt<T> s;
    s.h = tmax(wf - bf, (T)0);
    const IvC<T> ic = ivc(s.h, g, sqrtg, eps, hdry);
    s.u = ic.iv * Pf;
    s.v = ic.iv * Qf;
    s.c = ic.c;
    return s;
}

// Central-upwind flux from two face states; DIR 0: x-face, 1: y-face.
template <typename T, int DIR>
__device__ __forceinline__ void cu_flux_st(const FaceSt<T> &L, const FaceSt<T> &R, T g, T &H0, T &H1, T &H2)
{
    T unL = DIR == 0 ? L.u : L.v, unR = DIR == 0 ? R.u : R.v;
    T ap = tmax(tmax(unL + L.c, unR + R.c), (T)0);
    T am = tmin(tmin(unL - L.c, unR - R.c), (T)0);
    T den = ap - am;
    const bool moving = tlt((T)0, den);  // a+ = a- = 0: no flux
    T inv = trcp(moving ? den : (T)1);
    T pL = L.h * L.u, qL = L.h * L.v, pR = R.h * R.u, qR = R.h * R.v;
    T FL0, FL1, FL2, FR0, FR1, FR2;
    if (DIR == 0) {
        FL0 = pL; FL1 = pL * L.u + (T)0.5 * g * L.h * L.h; FL2 = qL * L.u;
        FR0 = pR; FR1 = pR * R.u + (T)0.5 * g * R.h * R.h; FR2 = qR * R.u;
    } else {
        FL0 = qL; FL1 = pL * L.v; FL2 = qL * L.v + (T)0.5 * g * L.h * L.h;
        FR0 = qR; FR1 = pR * R.v; FR2 = qR * R.v + (T)0.5 * g * R.h * R.h;
    }
    T k = ap * am * inv;
    H0 = moving ? (ap * FL0 - am * FR0) * inv + k * (R.h - L.h) : (T)0;
    H1 = moving ? (ap * FL1 - am * FR1) * inv + k * (pR - pL) : (T)0;
    H2 = moving ? (ap * FL2 - am * FR2) * inv + k * (qR - qL) : (T)0;
}

template <typename T>
__device__ __forceinline__ T shup(T v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
template <typename T>
__device__ __forceinline__ T shdn(T v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

constexpr int SW_COLS = 28;  // interior columns per warp strip (lanes 2..29)

// One warp walks a strip of 28 interior columns down ROWS rows.  Lane L holds
// column i = i0 - 2 + L.  Windows of rows live in registers: w, P, Q at rows
// r-3..r, eta at r-4..r, still depth at r-3..r, bed corners at r-2..r+1.  At
// step r the leading row r is loaded, the y-reconstruction of row r-1 and the
// y-face flux between rows r-2 and r-1 are formed, and row o = r-2 is finished:
// x-reconstruction and x-face flux (neighbours by shuffles), bed source,
// friction, dispersive differences (Eqs. 12-15) and the AB3 combine.  Every
// reconstruction and every face flux is computed once per strip.
// FAST: the default configuration fixed at compile time -- sequential cross
// form, compensated accumulation in single precision, no friction -- with
// both history levels always read (they hold zeros, weighted by zero, during
// the Euler start) and 32-bit offsets into the fields.
template <typename T, int ROWS, bool THETA1, bool FAST, int YS = 0>
__device__ __forceinline__ void rhs_sw_body(const Dev<T> &D, int blk, int nstrip)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    const int lane = threadIdx.x & 31;
    const int wg = blk * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int strip = wg % nstrip, band = wg / nstrip;
    const int nx = D.nx, ny = D.ny;
    const int j0 = band * ROWS;
    if (j0 >= ny) return;
    const int i = strip * SW_COLS - 2 + lane;           // this lane's column
    const int ic = min(i, nx + 1);                       // clamped for loads
    const int kc = min(i, nx + 2), kc1 = min(i + 1, nx + 2);
    const bool lane_out = lane >= 2 && lane <= 29 && i < nx;
    const T *w = D.w[cf.wc];
    const T g = D.g, eps = D.eps, hdry = D.hdry, th = THETA1 ? (T)1 : D.theta, sqrtg = tsqrt(g);
    const T rdx = D.rdx, rdy = D.rdy, half_rdx = (T)0.5 * rdx, half_rdy = (T)0.5 * rdy;
    const T rdx2 = rdx * rdx, rdy2 = rdy * rdy, q_rdxy = (T)0.25 * rdx * rdy;
    const T c_xxx = (T)0.5 * rdx2 * rdx, c_yyy = (T)0.5 * rdy2 * rdy;
    const T Bg = D.Bd * g, kB = D.Bd + (T)1 / (T)3, sixth = (T)1 / (T)6;
    const T b0c = coefv<T>(cf, 0, 0), b1c = coefv<T>(cf, 0, 1), b2c = coefv<T>(cf, 0, 2);
    const T g0c = coefv<T>(cf, 1, 0), g1c = coefv<T>(cf, 1, 1), g2c = coefv<T>(cf, 1, 2);
    const bool extrap = FAST ? false : D.cross_mode == 0;
    const bool kahan = FAST ? (sizeof(T) == 4) : (D.kahan != 0);
    const int nlev = FAST ? 3 : cf.nlev;
    const long long fs = D.fstride;
    T *H = D.hist;
    const T *corner = D.corner;
    const int cp = D.cpitch;

    // windows (index 3 = newest row)
    T wW[4] = {0, 0, 0, 0}, PW[4] = {0, 0, 0, 0}, QW[4] = {0, 0, 0, 0};
    T eW[5] = {0, 0, 0, 0, 0}, dW[4] = {0, 0, 0, 0}, bW[3] = {0, 0, 0};
    T KW[4] = {0, 0, 0, 0}, KRW[4] = {0, 0, 0, 0};  // corners at columns i and i+1, rows r-2..r+1
    FaceSt<T> Nprev = {0, 0, 0, 0};                  // N face state of row r-2
    T Hy0 = 0, Hy1 = 0, Hy2 = 0;                     // y-flux below row r-2 (face (r-2)-1/2)
    // passed on from the previous step: the y-differences q(r-1) - q(r-2) of
    // w, P, Q (the backward differences of this step's y-reconstruction), and
    // the face beds of the S and N faces of the previous reconstructed row
    // (this row's S face and the source's S face)
    T ayw = 0, ayP = 0, ayQ = 0, bSc = 0, bNc = 0;
    // eta_xx of the output row and the row below it, formed one and two steps
    // earlier as the eta_xx of the row above the output row
    T exx0 = 0, exx1 = 0;
    {
        int rr = min(j0 - 2, ny + 2);
        KW[3] = corner[(long long)(rr + 2) * cp + (kc + 2)];
        KRW[3] = corner[(long long)(rr + 2) * cp + (kc1 + 2)];
    }
    unsigned long long nclamp = 0;
    const int rend = min(j0 + ROWS, ny) + 2;
    // software pipeline: the leading row and the history of the next output
    // row are loaded one step ahead, so their latency overlaps the arithmetic
    // double precision also loads the bed at the centre, which set-up formed
    // from the same corners in the same order (bitwise what bed_centre gives
    // here), instead of twelve FP64 operations a cell
    constexpr bool BC_LOAD = sizeof(T) == 8;
    T pw, pP, pQ, pK, pKR, pB = (T)0;
    auto load_lead = [&](int r) {
        const int rr = min(r, ny + 1);
        const long long cr = fidx(D, ic, rr);
        const int kr = min(r + 1, ny + 2);
        pw = w[cr]; pP = D.P[cr]; pQ = D.Q[cr];
        if (BC_LOAD) pB = D.bC[cr];
        pK = corner[(long long)(kr + 2) * cp + (kc + 2)];
        pKR = corner[(long long)(kr + 2) * cp + (kc1 + 2)];
    };
    T hE1 = 0, hF1 = 0, hG1 = 0, hGs1 = 0, hFs1 = 0, hE2 = 0, hF2 = 0, hG2 = 0, hGs2 = 0, hFs2 = 0, hcw = 0;
    // YS > 0: the y-line chunk summaries of the three-launch y-solver (chunks of
    // YS rows) are formed here from the fresh dV, with the factors prefetched
    // with the history (what k_ysum computes from dV read back)
    T hym = 0, hye = 0, hyc = 0;
    T yt = 0, yPi = 1, yal0 = 0, yal1 = 0, ybe = 1;
    const int ynch = YS > 0 ? ychunk_stride((ny + YS - 1) / YS) : 0;
    const long long ys_s = (long long)nx * ynch;
    // 32-bit offsets of the history slots (FAST: the fields fit in 2^31 elements)
    const int ifs = (int)fs, s1o = cf.s1 * (int)fs, s2o = cf.s2 * (int)fs;
    auto load_hist = [&](int o) {
        if (lane_out && o >= j0 && o < ny) {
            if (FAST) {
                const int c = (o + 2) * D.pitch + i + D.hx;
                if (kahan) hcw = D.cw[c];
                if (YS > 0) { hym = D.fym[c]; hye = D.fye[c]; hyc = D.fyc[c]; }
                const T *h1 = H + (s1o + c), *h2 = H + (s2o + c);
                hE1 = h1[0]; hF1 = h1[3 * ifs]; hG1 = h1[6 * ifs]; hGs1 = h1[12 * ifs];
                hE2 = h2[0]; hF2 = h2[3 * ifs]; hG2 = h2[6 * ifs]; hGs2 = h2[12 * ifs];
                return;
            }
            const long long c = fidx(D, i, o);
            if (kahan) hcw = D.cw[c];
            if (nlev >= 2) {
                const long long oo = (long long)cf.s1 * fs + c;
                hE1 = H[0 * 3 * fs + oo]; hF1 = H[1 * 3 * fs + oo]; hG1 = H[2 * 3 * fs + oo]; hGs1 = H[4 * 3 * fs + oo];
                if (extrap) hFs1 = H[3 * 3 * fs + oo];
            }
            if (nlev >= 3) {
                const long long oo = (long long)cf.s2 * fs + c;
                hE2 = H[0 * 3 * fs + oo]; hF2 = H[1 * 3 * fs + oo]; hG2 = H[2 * 3 * fs + oo]; hGs2 = H[4 * 3 * fs + oo];
                if (extrap) hFs2 = H[3 * 3 * fs + oo];
            }
        }
    };
    load_lead(j0 - 2);
    for (int r = j0 - 2; r < rend; r++) {
        // ---- leading row r (prefetched), bed corners at row r+1
        T wn = pw, Pn = pP, Qn = pQ, Kn = pK, KRn = pKR, Bn = pB;
        T cE1 = hE1, cF1 = hF1, cG1 = hG1, cGs1 = hGs1, cFs1 = hFs1;
        T cE2 = hE2, cF2 = hF2, cG2 = hG2, cGs2 = hGs2, cFs2 = hFs2, ccw = hcw;
        const T cym = hym, cye = hye, cyc = hyc;
        if (r + 1 < rend) load_lead(r + 1);
        load_hist(r - 1);  // output row of the next step
#pragma unroll
        for (int q = 0; q < 3; q++) { wW[q] = wW[q + 1]; PW[q] = PW[q + 1]; QW[q] = QW[q + 1]; dW[q] = dW[q + 1]; KW[q] = KW[q + 1]; KRW[q] = KRW[q + 1]; }
#pragma unroll
        for (int q = 0; q < 4; q++) eW[q] = eW[q + 1];
        bW[0] = bW[1]; bW[1] = bW[2];
        wW[3] = wn; PW[3] = Pn; QW[3] = Qn; KW[3] = Kn; KRW[3] = KRn;
        // cell-centre bed of row r (mean of its 4 face values), d, eta
        {
            const T bc = BC_LOAD ? Bn : bed_centre(KW[2], KRW[2], KW[3], KRW[3]);
            T d = tmax(D.w_s - bc, (T)0);
            bW[2] = bc;
            dW[3] = d;
            eW[4] = tmax(wn - bc, (T)0) - d;
        }
        // ---- y-reconstruction of row r-1 (rows r-2, r-1, r) and the y-face flux
        //      between rows r-2 and r-1
        {
            const T bS = bNc, bN = (T)0.5 * (KW[2] + KRW[2]);
            const T bS0 = bSc, bN0 = bS;  // faces of the output row o = r - 2
            bSc = bS;
            bNc = bN;
            T wl, wh, Pl, Ph, Ql, Qh;
            if (THETA1) {
                const T cw = wW[3] - wW[2], cP = PW[3] - PW[2], cQ = QW[3] - QW[2];
                reconstruct_d(wW[2], ayw, cw, PW[2], ayP, cP, QW[2], ayQ, cQ, bS, bN, wl, wh, Pl, Ph, Ql, Qh);
                ayw = cw; ayP = cP; ayQ = cQ;
            } else {
                reconstruct(wW[1], wW[2], wW[3], PW[1], PW[2], PW[3], QW[1], QW[2], QW[3], bS, bN, th,
                            wl, wh, Pl, Ph, Ql, Qh);
            }
            FaceSt<T> S = face_state(wl, Pl, Ql, bS, g, sqrtg, eps, hdry);
            FaceSt<T> Nn = face_state(wh, Ph, Qh, bN, g, sqrtg, eps, hdry);
            T h0, h1, h2;
            cu_flux_st<T, 1>(Nprev, S, g, h0, h1, h2);  // face (r-1)-1/2 = o+1/2 for o = r-2
            // ---- finish row o = r - 2
            const int o = r - 2;
            // x-reconstruction of row o needs w, P, Q of the lanes next door
            // (lane 31 takes its own values where the lane to the right would
            // give them; nothing of lane 31 reaches an output lane)
            T w0 = wW[1], P0 = PW[1], Q0 = QW[1];
            T wp = shdn(w0, 1), Pm = shup(P0, 1), Pp = shdn(P0, 1);
            T Qm = shup(Q0, 1), Qp = shdn(Q0, 1);
            const T bxW = (T)0.5 * (KW[0] + KW[1]), bxE = shdn(bxW, 1);  // the E face is the next W face
            T xwl, xwh, xPl, xPh, xQl, xQh;
            if (THETA1) {
                const T cw = wp - w0, cP = Pp - P0, cQ = Qp - Q0;
                reconstruct_d(w0, shup(cw, 1), cw, P0, shup(cP, 1), cP, Q0, shup(cQ, 1), cQ, bxW, bxE, xwl, xwh, xPl,
                              xPh, xQl, xQh);
            } else {
                reconstruct(shup(w0, 1), w0, wp, Pm, P0, Pp, Qm, Q0, Qp, bxW, bxE, th, xwl, xwh, xPl, xPh, xQl, xQh);
            }
            FaceSt<T> Wst = face_state(xwl, xPl, xQl, bxW, g, sqrtg, eps, hdry);
            FaceSt<T> Est = face_state(xwh, xPh, xQh, bxE, g, sqrtg, eps, hdry);
            FaceSt<T> El;  // E state of the lane to the left
            El.h = shup(Est.h, 1); El.u = shup(Est.u, 1); El.v = shup(Est.v, 1); El.c = shup(Est.c, 1);
            T x0, x1, x2;
            cu_flux_st<T, 0>(El, Wst, g, x0, x1, x2);  // face i-1/2
            T xe0 = shdn(x0, 1), xe1 = shdn(x1, 1), xe2 = shdn(x2, 1);  // face i+1/2
            // neighbours for the dispersive and cross terms
            T em1 = shup(eW[2], 1), ep1 = shdn(eW[2], 1), em2 = shup(eW[2], 2), ep2 = shdn(eW[2], 2);
            T eSm = shup(eW[1], 1), eSp = shdn(eW[1], 1), eNm = shup(eW[3], 1), eNp = shdn(eW[3], 1);
            T dm = shup(dW[1], 1), dp = shdn(dW[1], 1);
            T QSm = shup(QW[0], 1), QSp = shdn(QW[0], 1), QNm = shup(QW[2], 1), QNp = shdn(QW[2], 1);
            T PSm = shup(PW[0], 1), PSp = shdn(PW[0], 1), PNm = shup(PW[2], 1), PNp = shdn(PW[2], 1);
            const bool valid = lane_out && o >= j0 && o < ny;
            {  // computed on every lane (no divergent region); stores predicated
                const long long c = fidx(D, i, o);
                T divx0 = (xe0 - x0) * rdx, divx1 = (xe1 - x1) * rdx, divx2 = (xe2 - x2) * rdx;
                T divy0 = (h0 - Hy0) * rdy, divy1 = (h1 - Hy1) * rdy, divy2 = (h2 - Hy2) * rdy;
                T bc = bW[0];
                // double precision reads the static terms set-up formed in the
                // same order of operations (the same values, bitwise)
                constexpr bool STAT = sizeof(T) == 8;
                // (the first two steps of a strip finish rows below the field's
                // halo, whose results are dropped: their reads stay in the field)
                const long long cst = STAT ? fidx(D, i, max(o, -2)) : 0;
                const T *st = STAT ? D.stat + cst : nullptr;
                const long long ss = STAT ? D.stat_stride : 0;
                T srcx, srcy;
                if constexpr (STAT) {
                    srcx = st[ST_SX * ss] * (w0 - st[ST_MX * ss]);
                    srcy = st[ST_SY * ss] * (w0 - st[ST_MY * ss]);
                } else {
                    srcx = -g * (bxE - bxW) * rdx * (w0 - (T)0.5 * (bxE + bxW));
                    srcy = -g * (bN0 - bS0) * rdy * (w0 - (T)0.5 * (bN0 + bS0));
                }
                T fr1 = (T)0, fr2 = (T)0;
                if (!FAST && D.friction != (T)0) {
                    T h = tmax(w0 - bc, (T)0);
                    T iv = (T)BSQ_SQRT2 * h * desing_inv(h, eps);
                    T u = iv * P0, v = iv * Q0;
                    T sp = tsqrt(u * u + v * v);
                    fr1 = D.friction * u * sp;
                    fr2 = D.friction * v * sp;
                }
                const T d = dW[1];
                T ddx, ddy, Bd2, Bd3;  // d_x, d_y, B g d^2, B g d^3
                if constexpr (STAT) {
                    ddx = st[ST_DDX * ss];
                    ddy = st[ST_DDY * ss];
                    Bd2 = st[ST_BD2 * ss];
                    Bd3 = st[ST_BD3 * ss];
                } else {
                    ddx = (dp - dm) * half_rdx;
                    ddy = (dW[2] - dW[0]) * half_rdy;
                    Bd2 = Bg * d * d;
                    Bd3 = Bd2 * d;
                }
                const T e0 = eW[2];
                // eta_xx of rows o-1, o, o+1: two passed on, one new; eta_yy of
                // the lanes next door by shuffles (the same expressions, so the
                // same values)
                const T exx_p = (eNp - (T)2 * eW[3] + eNm) * rdx2;
                const T e_xx = exx0, exx_m = exx1;
                exx1 = exx0;
                exx0 = exx_p;
                T e_yy = (eW[3] - (T)2 * e0 + eW[1]) * rdy2;
                T e_xy = (eNp - eSp - eNm + eSm) * q_rdxy;
                T e_xxx = (ep2 - (T)2 * ep1 + (T)2 * em1 - em2) * c_xxx;
                T e_yyy = (eW[4] - (T)2 * eW[3] + (T)2 * eW[1] - eW[0]) * c_yyy;
                const T eyy_p = shdn(e_yy, 1), eyy_m = shup(e_yy, 1);
                T e_xyy = (eyy_p - eyy_m) * half_rdx;
                T e_xxy = (exx_p - exx_m) * half_rdy;
                T dispx = Bd3 * (e_xxx + e_xyy) + Bd2 * (ddx * ((T)2 * e_xx + e_yy) + ddy * e_xy);
                T dispy = Bd3 * (e_yyy + e_xxy) + Bd2 * (ddy * ((T)2 * e_yy + e_xx) + ddx * e_xy);
                T E = -divx0 - divy0;
                T F = -divx1 - divy1 + srcx - fr1 + dispx;
                T G = -divx2 - divy2 + srcy - fr2 + dispy;
                T Q_x = (Qp - Qm) * half_rdx;
                T Q_y = (QW[2] - QW[0]) * half_rdy;
                T Q_xy = (QNp - QSp - QNm + QSm) * q_rdxy;
                T P_x = (Pp - Pm) * half_rdx;
                T P_y = (PW[2] - PW[0]) * half_rdy;
                T P_xy = (PNp - PSp - PNm + PSm) * q_rdxy;
                T Fs, Gs;
                if constexpr (sizeof(T) == 8) {
                    const T c1 = D.fsc1[cst], c2 = D.fsc2[cst], c3 = D.fsc3[cst];
                    Fs = c1 * Q_y + c2 * Q_x + c3 * Q_xy;
                    Gs = c2 * P_x + c1 * P_y + c3 * P_xy;
                } else {
                    Fs = d * ddx * Q_y * sixth + d * ddy * Q_x * sixth + kB * d * d * Q_xy;
                    Gs = d * ddy * P_x * sixth + d * ddx * P_y * sixth + kB * d * d * P_xy;
                }
                // AB3 / Euler combine (Eqs. 42-43), history prefetched one step ahead
                T dw = b0c * E, dU = b0c * F, dV = b0c * G + g0c * Gs;
                if (extrap) dU += g0c * Fs;
                if (nlev >= 2) {
                    dw += b1c * cE1;
                    dU += b1c * cF1;
                    dV += b1c * cG1 + g1c * cGs1;
                    if (extrap) dU += g1c * cFs1;
                }
                if (nlev >= 3) {
                    dw += b2c * cE2;
                    dU += b2c * cF2;
                    dV += b2c * cG2 + g2c * cGs2;
                    if (extrap) dU += g2c * cFs2;
                }
                if (!extrap) dU -= Fs;
                if (FAST) {
                    const int ci = (o + 2) * D.pitch + i + D.hx;
                    const T y = kahan ? dw - ccw : dw;
                    T wnew = w0 + y;
                    T cwn = kahan ? (wnew - w0) - y : (T)0;
                    const bool cl = tlt(wnew, bc);
                    wnew = cl ? bc : wnew;
                    cwn = cl ? (T)0 : cwn;
                    nclamp += (valid && cl) ? 1ull : 0ull;
                    if (valid) {
                        T *h0 = H + (cf.s0 * ifs + ci);
                        h0[0] = E; h0[3 * ifs] = F; h0[6 * ifs] = G; h0[12 * ifs] = Gs;
                        D.w[cf.wc ^ 1][ci] = wnew;
                        if (kahan) D.cw[ci] = cwn;
                        D.dU[ci] = dU;
                        D.dV[ci] = dV;
                        if (YS > 0) {
                            // same recurrences as k_ysum, row by row
                            T rr = dV;
                            if (o == 0) rr += D.corrS[i];
                            if (o == ny - 1) rr += D.corrN[i];
                            yt = cym * rr + cye * yt;
                            yPi = cye * yPi;
                            yal0 = yal0 + ybe * yt;
                            yal1 = yal1 + ybe * yPi;
                            ybe = -cyc * ybe;
                            if ((o + 1) % YS == 0 || o == ny - 1) {
                                const long long so = (long long)i * ynch + o / YS;
                                T *sums = D.ysums;
                                sums[so] = yPi;
                                sums[ys_s + so] = yt;
                                sums[2 * ys_s + so] = yal0;
                                sums[3 * ys_s + so] = yal1;
                                sums[4 * ys_s + so] = ybe;
                                yt = 0; yPi = 1; yal0 = 0; yal1 = 0; ybe = 1;
                            }
                        }
                    }
                } else if (valid) {
                {
                    const long long oo = (long long)cf.s0 * fs + c;
                    H[0 * 3 * fs + oo] = E;
                    H[1 * 3 * fs + oo] = F;
                    H[2 * 3 * fs + oo] = G;
                    if (extrap) H[3 * 3 * fs + oo] = Fs;
                    H[4 * 3 * fs + oo] = Gs;
                }
                T wnew, cwn = (T)0;
                if (kahan) {
                    T y = dw - ccw;
                    wnew = w0 + y;
                    cwn = (wnew - w0) - y;
                } else {
                    wnew = w0 + dw;
                }
                if (tlt(wnew, bc)) { wnew = bc; cwn = (T)0; nclamp++; }
                D.w[cf.wc ^ 1][c] = wnew;
                if (kahan) D.cw[c] = cwn;
                D.dU[c] = dU;
                D.dV[c] = dV;
                }
            }
            Nprev = Nn;
            Hy0 = h0; Hy1 = h1; Hy2 = h2;
        }
    }
    // positivity clamps: warp total, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) nclamp += __shfl_xor_sync(0xffffffffu, nclamp, o);
    if (lane == 0 && nclamp) atomicAdd(&D.ctl->clamps, nclamp);
    if (blk == 0 && threadIdx.x == 0) {
        // commit the step in the controller state (the controller kernel of
        // this step has finished; no thread of this kernel reads Ctl)
        Ctl *ct = D.ctl;
        ct->dtm2 = ct->dtm1;
        ct->dtm1 = cf.dt;
        ct->last_dt = cf.dt;
        ct->t = cf.t1;
        ct->n = cf.n + 1;
        ct->rate_bits = 0ull;
    }
}

template <typename T, int ROWS, bool THETA1, bool FAST, int YS = 0>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2) k_rhs_sw(Dev<T> D, int nstrip)
{
    rhs_sw_body<T, ROWS, THETA1, FAST, YS>(D, blockIdx.x, nstrip);
}

// ------------------------------------------------------------------ RHS + combine, two columns per lane
//
// Single precision, default configuration (theta = 1, sequential cross form,
// compensated accumulation, no friction).  Lane L of a warp holds the two
// adjacent columns c0 = base + 2L and c0 + 1 of a strip of 60 interior columns
// (lanes 1..30; lanes 0 and 31 are the 2-column halo on each side) and walks
// ROWS rows like k_rhs_sw.  Both columns go through the same arithmetic, so
// it is done on pairs with the packed single-precision instructions (two
// results per add, multiply or fused multiply-add); comparisons, selects,
// square roots and reciprocals stay per column.  A lane's x-neighbours come
// from its own pair and the pairs of lanes L-1 and L+1.  Same arithmetic as
// k_rhs_sw up to the fusion of multiply-adds.

typedef float2 f2;
__device__ __forceinline__ f2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 sc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, sc2(-1.0f), a); }  // exact a - b
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 max2(f2 a, f2 b) { return mk2(tmax(a.x, b.x), tmax(a.y, b.y)); }
__device__ __forceinline__ f2 min2(f2 a, f2 b) { return mk2(tmin(a.x, b.x), tmin(a.y, b.y)); }
__device__ __forceinline__ f2 up2(f2 v) { return mk2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1)); }
__device__ __forceinline__ f2 dn2(f2 v) { return mk2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1)); }
__device__ __forceinline__ f2 ld2(const float *p) { return *reinterpret_cast<const f2 *>(p); }
__device__ __forceinline__ void st2(float *p, f2 v) { *reinterpret_cast<f2 *>(p) = v; }

// minmod(a, c) = max(min(a, c), 0) + min(max(a, c), 0): at most one of the
// two terms is nonzero (the smaller of two positive differences, the larger
// of two negative ones, else 0), so the sum is exact and branch free.
__device__ __forceinline__ f2 slope2(f2 m, f2 z, f2 p)
{
    const f2 a = sub2(z, m), c = sub2(p, z);
    const f2 lo = max2(min2(a, c), sc2(0.0f)), hi = min2(max2(a, c), sc2(0.0f));
    return add2(lo, hi);
}
// reconstruction of one variable: low / high face values
__device__ __forceinline__ void recon_pair(f2 m, f2 z, f2 p, f2 &lo, f2 &hi)
{
    const f2 s = slope2(m, z, p);
    lo = fma2(sc2(-0.5f), s, z);
    hi = fma2(sc2(0.5f), s, z);
}
// water level with the positivity fix against the face beds blo, bhi.  The
// cell mean is not below the mean of its two face beds (the update clamps
// w >= b at the centre, which is that mean), so at most one face value lies
// below its bed: the face below its bed is raised to it and the other face
// takes the difference, keeping the sum of the two (2 w): with
//   delta = max(bhi - hi, 0) - max(blo - lo, 0),
// hi += delta and lo -= delta, branch free.
__device__ __forceinline__ void recon_w_pair(f2 m, f2 z, f2 p, f2 blo, f2 bhi, f2 &lo, f2 &hi)
{
    const f2 s = slope2(m, z, p);
    const f2 a = fma2(sc2(0.5f), s, z), b = fma2(sc2(-0.5f), s, z);
    const f2 delta = sub2(max2(sub2(bhi, a), sc2(0.0f)), max2(sub2(blo, b), sc2(0.0f)));
    hi = add2(a, delta);
    lo = sub2(b, delta);
}

struct FS2 {
    f2 h, u, v, c;
};
__device__ __forceinline__ FS2 face_pair(f2 wf, f2 Pf, f2 Qf, f2 bf, float g, float eps)
{
    FS2 s;
    s.h = max2(sub2(wf, bf), sc2(0.0f));
    const f2 h2 = mul2(s.h, s.h), h4 = mul2(h2, h2);
    const f2 den = add2(h4, max2(h4, sc2(eps)));
    const f2 iv = mul2(mul2(sc2((float)BSQ_SQRT2), s.h), mk2(trsqrt(den.x), trsqrt(den.y)));
    s.u = mul2(iv, Pf);
    s.v = mul2(iv, Qf);
    const f2 gh = mul2(sc2(g), s.h);
    s.c = mk2(tsqrt(gh.x), tsqrt(gh.y));
    return s;
}
// central-upwind flux (Eq. 5) on a pair of faces of one direction
template <int DIR>
__device__ __forceinline__ void flux_pair(const FS2 &L, const FS2 &R, float g, f2 &H0, f2 &H1, f2 &H2)
{
    const f2 unL = DIR == 0 ? L.u : L.v, unR = DIR == 0 ? R.u : R.v;
    const f2 ap = max2(max2(add2(unL, L.c), add2(unR, R.c)), sc2(0.0f));
    const f2 am = min2(min2(sub2(unL, L.c), sub2(unR, R.c)), sc2(0.0f));
    // a+ = a- = 0 (both sides dry): with den floored at 1e-30 every term below
    // is an exact zero, which is the flux of Eq. 5 in that case
    const f2 den = max2(sub2(ap, am), sc2(1e-30f));
    const f2 inv = mk2(trcp(den.x), trcp(den.y));
    const f2 pL = mul2(L.h, L.u), qL = mul2(L.h, L.v), pR = mul2(R.h, R.u), qR = mul2(R.h, R.v);
    const f2 hg = sc2(0.5f * g);
    const f2 hhL = mul2(mul2(hg, L.h), L.h), hhR = mul2(mul2(hg, R.h), R.h);
    f2 FL0, FL1, FL2, FR0, FR1, FR2;
    if (DIR == 0) {
        FL0 = pL; FL1 = fma2(pL, L.u, hhL); FL2 = mul2(qL, L.u);
        FR0 = pR; FR1 = fma2(pR, R.u, hhR); FR2 = mul2(qR, R.u);
    } else {
        FL0 = qL; FL1 = mul2(pL, L.v); FL2 = fma2(qL, L.v, hhL);
        FR0 = qR; FR1 = mul2(pR, R.v); FR2 = fma2(qR, R.v, hhR);
    }
    const f2 k = mul2(mul2(ap, am), inv);
    const f2 nam = mul2(am, sc2(-1.0f));
    const f2 t0 = fma2(k, sub2(R.h, L.h), mul2(fma2(nam, FR0, mul2(ap, FL0)), inv));
    const f2 t1 = fma2(k, sub2(pR, pL), mul2(fma2(nam, FR1, mul2(ap, FL1)), inv));
    const f2 t2 = fma2(k, sub2(qR, qL), mul2(fma2(nam, FR2, mul2(ap, FL2)), inv));
    H0 = t0;
    H1 = t1;
    H2 = t2;
}

constexpr int SW2_COLS = 60;  // interior columns per warp strip (two per lane, lanes 1..30)

// FRIC: quadratic bottom friction f1 = f u |u|, f2 = f v |u| in F and G, with
// the desingularised centre velocities (the paper names the quadratic law and
// f = 0.0025 in Sec. 5.4 without writing it out)
template <int YS, bool FRIC = false>
__device__ __forceinline__ void rhs_sw2_body(const Dev<float> &D, int blk, int nstrip, int ROWS)
{
    typedef float T;
    const Coef cf = *D.coef;
    if (!cf.active) return;
    const int lane = threadIdx.x & 31;
    const int wg = blk * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int strip = wg % nstrip, band = wg / nstrip;
    const int nx = D.nx, ny = D.ny;
    const int j0 = band * ROWS;
    if (j0 >= ny) return;
    const int c0 = strip * SW2_COLS - 2 + 2 * lane;  // this lane's columns c0, c0 + 1
    const bool inner = lane >= 1 && lane <= 30;
    const bool out0 = inner && c0 < nx, out1 = inner && c0 + 1 < nx;
    const int kc0 = min(c0, nx + 2), kc1 = min(c0 + 1, nx + 2), kc2 = min(c0 + 2, nx + 2);
    const T *w = D.w[cf.wc];
    const float g = D.g, eps = D.eps;
    const float rdx = D.rdx, rdy = D.rdy;
    const float half_rdx = 0.5f * rdx, half_rdy = 0.5f * rdy;
    const float rdx2 = rdx * rdx, rdy2 = rdy * rdy, q_rdxy = 0.25f * rdx * rdy;
    const float c_xxx = 0.5f * rdx2 * rdx, c_yyy = 0.5f * rdy2 * rdy;
    const float Bg = D.Bd * g, kB = D.Bd + 1.0f / 3.0f, sixth = 1.0f / 6.0f;
    const float b0c = cf.betaf[0], b1c = cf.betaf[1], b2c = cf.betaf[2];
    const float g0c = cf.gamf[0], g1c = cf.gamf[1], g2c = cf.gamf[2];
    T *H = D.hist;
    const T *corner = D.corner;
    const int cp = D.cpitch;
    const int pitch = D.pitch, hx = D.hx;
    const int ifs = (int)D.fstride, s0o = cf.s0 * ifs, s1o = cf.s1 * ifs, s2o = cf.s2 * ifs;

    f2 wW[4], PW[4], QW[4], eW[5], dW[4], bW[3], KW[4], KRW[4];
#pragma unroll
    for (int q = 0; q < 5; q++) eW[q] = sc2(0.0f);
#pragma unroll
    for (int q = 0; q < 4; q++) { wW[q] = PW[q] = QW[q] = dW[q] = KW[q] = KRW[q] = sc2(0.0f); }
#pragma unroll
    for (int q = 0; q < 3; q++) bW[q] = sc2(0.0f);
    FS2 Nprev = {sc2(0.0f), sc2(0.0f), sc2(0.0f), sc2(0.0f)};
    f2 Hy0 = sc2(0.0f), Hy1 = sc2(0.0f), Hy2 = sc2(0.0f);
    {
        const int rr = min(j0 - 2, ny + 2);
        const T *kr = corner + (long long)(rr + 2) * cp + 2;
        const float k0 = kr[kc0], k1 = kr[kc1], k2 = kr[kc2];
        KW[3] = mk2(k0, k1);
        KRW[3] = mk2(k1, k2);
    }
    unsigned long long nclamp = 0;
    const int rend = min(j0 + ROWS, ny) + 2;
    f2 pw, pP, pQ, pK, pKR;
    auto load_lead = [&](int r) {
        const int rr = min(r, ny + 1);
        const int cr = (rr + 2) * pitch + c0 + hx;
        pw = ld2(w + cr); pP = ld2(D.P + cr); pQ = ld2(D.Q + cr);
        const int kr = min(r + 1, ny + 2);
        const T *kp = corner + (long long)(kr + 2) * cp + 2;
        const float k0 = kp[kc0], k1 = kp[kc1], k2 = kp[kc2];
        pK = mk2(k0, k1);
        pKR = mk2(k1, k2);
    };
    f2 hE1 = sc2(0.0f), hF1 = hE1, hG1 = hE1, hGs1 = hE1, hE2 = hE1, hF2 = hE1, hG2 = hE1, hGs2 = hE1, hcw = hE1;
    f2 hym = hE1, hye = hE1, hyc = hE1;
    f2 yt = sc2(0.0f), yPi = sc2(1.0f), yal0 = sc2(0.0f), yal1 = sc2(0.0f), ybe = sc2(1.0f);
    const int ynch = YS > 0 ? ychunk_stride((ny + YS - 1) / YS) : 0;
    const long long ys_s = (long long)nx * ynch;
    auto load_hist = [&](int o) {
        if (out0 && o >= j0 && o < ny) {
            const int c = (o + 2) * pitch + c0 + hx;
            hcw = ld2(D.cw + c);
            const T *h1 = H + (s1o + c), *h2 = H + (s2o + c);
            hE1 = ld2(h1); hF1 = ld2(h1 + 3 * ifs); hG1 = ld2(h1 + 6 * ifs); hGs1 = ld2(h1 + 12 * ifs);
            hE2 = ld2(h2); hF2 = ld2(h2 + 3 * ifs); hG2 = ld2(h2 + 6 * ifs); hGs2 = ld2(h2 + 12 * ifs);
            if (YS > 0) { hym = ld2(D.fym + c); hye = ld2(D.fye + c); hyc = ld2(D.fyc + c); }
        }
    };
    load_lead(j0 - 2);
    for (int r = j0 - 2; r < rend; r++) {
        const f2 wn = pw, Pn = pP, Qn = pQ, Kn = pK, KRn = pKR;
        const f2 cE1 = hE1, cF1 = hF1, cG1 = hG1, cGs1 = hGs1, cE2 = hE2, cF2 = hF2, cG2 = hG2, cGs2 = hGs2;
        const f2 ccw = hcw, cym = hym, cye = hye, cyc = hyc;
        if (r + 1 < rend) load_lead(r + 1);
        load_hist(r - 1);
#pragma unroll
        for (int q = 0; q < 3; q++) { wW[q] = wW[q + 1]; PW[q] = PW[q + 1]; QW[q] = QW[q + 1]; dW[q] = dW[q + 1]; KW[q] = KW[q + 1]; KRW[q] = KRW[q + 1]; }
#pragma unroll
        for (int q = 0; q < 4; q++) eW[q] = eW[q + 1];
        bW[0] = bW[1]; bW[1] = bW[2];
        wW[3] = wn; PW[3] = Pn; QW[3] = Qn; KW[3] = Kn; KRW[3] = KRn;
        {
            const f2 half = sc2(0.5f);
            const f2 bw_ = mul2(half, add2(KW[2], KW[3])), be_ = mul2(half, add2(KRW[2], KRW[3]));
            const f2 bs_ = mul2(half, add2(KW[2], KRW[2])), bn_ = mul2(half, add2(KW[3], KRW[3]));
            const f2 bc = mul2(sc2(0.25f), add2(add2(add2(bw_, be_), bs_), bn_));
            const f2 d = max2(sub2(sc2(D.w_s), bc), sc2(0.0f));
            bW[2] = bc;
            dW[3] = d;
            eW[4] = sub2(max2(sub2(wn, bc), sc2(0.0f)), d);
        }
        // y-reconstruction of row r-1, y-face flux between rows r-2 and r-1
        const f2 bS = mul2(sc2(0.5f), add2(KW[1], KRW[1])), bN = mul2(sc2(0.5f), add2(KW[2], KRW[2]));
        f2 wl, wh, Pl, Ph, Ql, Qh;
        recon_w_pair(wW[1], wW[2], wW[3], bS, bN, wl, wh);
        recon_pair(PW[1], PW[2], PW[3], Pl, Ph);
        recon_pair(QW[1], QW[2], QW[3], Ql, Qh);
        const FS2 S = face_pair(wl, Pl, Ql, bS, g, eps);
        const FS2 Nn = face_pair(wh, Ph, Qh, bN, g, eps);
        f2 h0, h1, h2;
        flux_pair<1>(Nprev, S, g, h0, h1, h2);
        // ---- finish row o = r - 2
        const int o = r - 2;
        const f2 w0 = wW[1], P0 = PW[1], Q0 = QW[1];
        // x-neighbours: own pair and the pairs of lanes L-1 (m) and L+1 (p)
        const f2 wLm = up2(w0), wLp = dn2(w0), PLm = up2(P0), PLp = dn2(P0), QLm = up2(Q0), QLp = dn2(Q0);
        const f2 wm = mk2(wLm.y, w0.x), wp = mk2(w0.y, wLp.x);
        const f2 Pm = mk2(PLm.y, P0.x), Pp = mk2(P0.y, PLp.x);
        const f2 Qm = mk2(QLm.y, Q0.x), Qp = mk2(Q0.y, QLp.x);
        const f2 bxW = mul2(sc2(0.5f), add2(KW[0], KW[1])), bxE = mul2(sc2(0.5f), add2(KRW[0], KRW[1]));
        f2 xwl, xwh, xPl, xPh, xQl, xQh;
        recon_w_pair(wm, w0, wp, bxW, bxE, xwl, xwh);
        recon_pair(Pm, P0, Pp, xPl, xPh);
        recon_pair(Qm, Q0, Qp, xQl, xQh);
        const FS2 Wst = face_pair(xwl, xPl, xQl, bxW, g, eps);
        const FS2 Est = face_pair(xwh, xPh, xQh, bxE, g, eps);
        // E state of the column to the left: lane L-1's second column, own first
        FS2 El;
        El.h = mk2(__shfl_up_sync(0xffffffffu, Est.h.y, 1), Est.h.x);
        El.u = mk2(__shfl_up_sync(0xffffffffu, Est.u.y, 1), Est.u.x);
        El.v = mk2(__shfl_up_sync(0xffffffffu, Est.v.y, 1), Est.v.x);
        El.c = mk2(__shfl_up_sync(0xffffffffu, Est.c.y, 1), Est.c.x);
        f2 x0, x1, x2;
        flux_pair<0>(El, Wst, g, x0, x1, x2);  // faces c - 1/2
        const f2 xe0 = mk2(x0.y, __shfl_down_sync(0xffffffffu, x0.x, 1));  // faces c + 1/2
        const f2 xe1 = mk2(x1.y, __shfl_down_sync(0xffffffffu, x1.x, 1));
        const f2 xe2 = mk2(x2.y, __shfl_down_sync(0xffffffffu, x2.x, 1));
        // neighbours for the dispersive and cross terms
        const f2 e0 = eW[2];
        const f2 eLm = up2(e0), eLp = dn2(e0);
        const f2 em1 = mk2(eLm.y, e0.x), ep1 = mk2(e0.y, eLp.x), em2 = eLm, ep2 = eLp;
        const f2 eS = eW[1], eN = eW[3];
        const float eSLm = __shfl_up_sync(0xffffffffu, eS.y, 1), eSLp = __shfl_down_sync(0xffffffffu, eS.x, 1);
        const float eNLm = __shfl_up_sync(0xffffffffu, eN.y, 1), eNLp = __shfl_down_sync(0xffffffffu, eN.x, 1);
        const f2 eSm = mk2(eSLm, eS.x), eSp = mk2(eS.y, eSLp), eNm = mk2(eNLm, eN.x), eNp = mk2(eN.y, eNLp);
        const f2 dd = dW[1];
        const f2 dm = mk2(__shfl_up_sync(0xffffffffu, dd.y, 1), dd.x), dp = mk2(dd.y, __shfl_down_sync(0xffffffffu, dd.x, 1));
        const f2 QS = QW[0], QN = QW[2], PS = PW[0], PN = PW[2];
        const f2 QSm = mk2(__shfl_up_sync(0xffffffffu, QS.y, 1), QS.x), QSp = mk2(QS.y, __shfl_down_sync(0xffffffffu, QS.x, 1));
        const f2 QNm = mk2(__shfl_up_sync(0xffffffffu, QN.y, 1), QN.x), QNp = mk2(QN.y, __shfl_down_sync(0xffffffffu, QN.x, 1));
        const f2 PSm = mk2(__shfl_up_sync(0xffffffffu, PS.y, 1), PS.x), PSp = mk2(PS.y, __shfl_down_sync(0xffffffffu, PS.x, 1));
        const f2 PNm = mk2(__shfl_up_sync(0xffffffffu, PN.y, 1), PN.x), PNp = mk2(PN.y, __shfl_down_sync(0xffffffffu, PN.x, 1));
        const bool valid = (out0 || out1) && o >= j0 && o < ny;
        {
            const f2 srdx = sc2(rdx), srdy = sc2(rdy);
            const f2 divx0 = mul2(sub2(xe0, x0), srdx), divx1 = mul2(sub2(xe1, x1), srdx), divx2 = mul2(sub2(xe2, x2), srdx);
            const f2 divy0 = mul2(sub2(h0, Hy0), srdy), divy1 = mul2(sub2(h1, Hy1), srdy), divy2 = mul2(sub2(h2, Hy2), srdy);
            const f2 bS0 = mul2(sc2(0.5f), add2(KW[0], KRW[0])), bN0 = mul2(sc2(0.5f), add2(KW[1], KRW[1]));
            const f2 bc = bW[0];
            const f2 ng = sc2(-g);
            const f2 srcx = mul2(mul2(mul2(ng, sub2(bxE, bxW)), srdx), fma2(sc2(-0.5f), add2(bxE, bxW), w0));
            const f2 srcy = mul2(mul2(mul2(ng, sub2(bN0, bS0)), srdy), fma2(sc2(-0.5f), add2(bN0, bS0), w0));
            const f2 d = dd;
            const f2 ddx = mul2(sub2(dp, dm), sc2(half_rdx));
            const f2 ddy = mul2(sub2(dW[2], dW[0]), sc2(half_rdy));
            const f2 m2 = sc2(-2.0f), p2 = sc2(2.0f);
            const f2 e_xx = mul2(add2(fma2(m2, e0, ep1), em1), sc2(rdx2));
            const f2 e_yy = mul2(add2(fma2(m2, e0, eW[3]), eW[1]), sc2(rdy2));
            const f2 e_xy = mul2(add2(sub2(sub2(eNp, eSp), eNm), eSm), sc2(q_rdxy));
            const f2 e_xxx = mul2(sub2(fma2(p2, em1, fma2(m2, ep1, ep2)), em2), sc2(c_xxx));
            const f2 e_yyy = mul2(sub2(fma2(p2, eW[1], fma2(m2, eW[3], eW[4])), eW[0]), sc2(c_yyy));
            const f2 eyy_p = mul2(add2(fma2(m2, ep1, eNp), eSp), sc2(rdy2));
            const f2 eyy_m = mul2(add2(fma2(m2, em1, eNm), eSm), sc2(rdy2));
            const f2 exx_p = mul2(add2(fma2(m2, eW[3], eNp), eNm), sc2(rdx2));
            const f2 exx_m = mul2(add2(fma2(m2, eW[1], eSp), eSm), sc2(rdx2));
            const f2 e_xyy = mul2(sub2(eyy_p, eyy_m), sc2(half_rdx));
            const f2 e_xxy = mul2(sub2(exx_p, exx_m), sc2(half_rdy));
            const f2 Bgd2 = mul2(mul2(sc2(Bg), d), d), Bgd3 = mul2(Bgd2, d);
            const f2 dispx = fma2(Bgd3, add2(e_xxx, e_xyy), mul2(Bgd2, fma2(ddx, fma2(p2, e_xx, e_yy), mul2(ddy, e_xy))));
            const f2 dispy = fma2(Bgd3, add2(e_yyy, e_xxy), mul2(Bgd2, fma2(ddy, fma2(p2, e_yy, e_xx), mul2(ddx, e_xy))));
            const f2 E = sub2(mul2(divx0, sc2(-1.0f)), divy0);
            f2 F = add2(add2(sub2(mul2(divx1, sc2(-1.0f)), divy1), srcx), dispx);
            f2 G = add2(add2(sub2(mul2(divx2, sc2(-1.0f)), divy2), srcy), dispy);
            if (FRIC) {
                const f2 h = max2(sub2(w0, bc), sc2(0.0f));
                const f2 h2 = mul2(h, h), h4 = mul2(h2, h2);
                const f2 den = add2(h4, max2(h4, sc2(eps)));
                const f2 iv = mul2(mul2(sc2((float)BSQ_SQRT2), h), mk2(trsqrt(den.x), trsqrt(den.y)));
                const f2 u = mul2(iv, P0), v = mul2(iv, Q0);
                const f2 sp2 = fma2(u, u, mul2(v, v));
                const f2 fsp = mul2(sc2(D.friction), mk2(tsqrt(sp2.x), tsqrt(sp2.y)));
                F = sub2(F, mul2(fsp, u));
                G = sub2(G, mul2(fsp, v));
            }
            const f2 Q_x = mul2(sub2(Qp, Qm), sc2(half_rdx));
            const f2 Q_y = mul2(sub2(QW[2], QW[0]), sc2(half_rdy));
            const f2 Q_xy = mul2(add2(sub2(sub2(QNp, QSp), QNm), QSm), sc2(q_rdxy));
            const f2 P_x = mul2(sub2(Pp, Pm), sc2(half_rdx));
            const f2 P_y = mul2(sub2(PW[2], PW[0]), sc2(half_rdy));
            const f2 P_xy = mul2(add2(sub2(sub2(PNp, PSp), PNm), PSm), sc2(q_rdxy));
            const f2 dsx = mul2(mul2(d, ddx), sc2(sixth)), dsy = mul2(mul2(d, ddy), sc2(sixth));
            const f2 kBd2 = mul2(mul2(sc2(kB), d), d);
            const f2 Fs = fma2(kBd2, Q_xy, fma2(dsy, Q_x, mul2(dsx, Q_y)));
            const f2 Gs = fma2(kBd2, P_xy, fma2(dsx, P_y, mul2(dsy, P_x)));
            // AB3 / Euler combine (Eqs. 42-43), both history levels read
            f2 dw = mul2(sc2(b0c), E), dU = mul2(sc2(b0c), F), dV = fma2(sc2(g0c), Gs, mul2(sc2(b0c), G));
            dw = fma2(sc2(b1c), cE1, dw);
            dU = fma2(sc2(b1c), cF1, dU);
            dV = add2(dV, fma2(sc2(g1c), cGs1, mul2(sc2(b1c), cG1)));
            dw = fma2(sc2(b2c), cE2, dw);
            dU = fma2(sc2(b2c), cF2, dU);
            dV = add2(dV, fma2(sc2(g2c), cGs2, mul2(sc2(b2c), cG2)));
            dU = sub2(dU, Fs);  // F*(Q^{n+1}) is added by the x-line kernel
            const f2 y = sub2(dw, ccw);
            f2 wnew = add2(w0, y);
            f2 cwn = sub2(sub2(wnew, w0), y);
            const bool clx = wnew.x < bc.x, cly = wnew.y < bc.y;
            wnew = mk2(clx ? bc.x : wnew.x, cly ? bc.y : wnew.y);
            cwn = mk2(clx ? 0.0f : cwn.x, cly ? 0.0f : cwn.y);
            nclamp += (valid && out0 && clx ? 1ull : 0ull) + (valid && out1 && cly ? 1ull : 0ull);
            if (valid) {
                const int ci = (o + 2) * pitch + c0 + hx;
                T *hp = H + (s0o + ci);
                T *wp_ = D.w[cf.wc ^ 1] + ci;
                if (out1) {
                    st2(hp, E); st2(hp + 3 * ifs, F); st2(hp + 6 * ifs, G); st2(hp + 12 * ifs, Gs);
                    st2(wp_, wnew); st2(D.cw + ci, cwn); st2(D.dU + ci, dU); st2(D.dV + ci, dV);
                } else {
                    hp[0] = E.x; hp[3 * ifs] = F.x; hp[6 * ifs] = G.x; hp[12 * ifs] = Gs.x;
                    *wp_ = wnew.x; D.cw[ci] = cwn.x; D.dU[ci] = dU.x; D.dV[ci] = dV.x;
                }
                if (YS > 0) {
                    // the chunk summaries of k_ysum, per column
                    f2 rr = dV;
                    if (o == 0) rr = add2(rr, mk2(D.corrS[c0], out1 ? D.corrS[c0 + 1] : 0.0f));
                    if (o == ny - 1) rr = add2(rr, mk2(D.corrN[c0], out1 ? D.corrN[c0 + 1] : 0.0f));
                    yt = fma2(cym, rr, mul2(cye, yt));
                    yPi = mul2(cye, yPi);
                    yal0 = fma2(ybe, yt, yal0);
                    yal1 = fma2(ybe, yPi, yal1);
                    ybe = mul2(mul2(cyc, sc2(-1.0f)), ybe);
                    if ((o + 1) % YS == 0 || o == ny - 1) {
                        const int kk = o / YS;
                        T *sums = D.ysums;
                        const long long so0 = (long long)c0 * ynch + kk;
                        sums[so0] = yPi.x; sums[ys_s + so0] = yt.x; sums[2 * ys_s + so0] = yal0.x;
                        sums[3 * ys_s + so0] = yal1.x; sums[4 * ys_s + so0] = ybe.x;
                        if (out1) {
                            const long long so1 = so0 + ynch;
                            sums[so1] = yPi.y; sums[ys_s + so1] = yt.y; sums[2 * ys_s + so1] = yal0.y;
                            sums[3 * ys_s + so1] = yal1.y; sums[4 * ys_s + so1] = ybe.y;
                        }
                        yt = sc2(0.0f); yPi = sc2(1.0f); yal0 = sc2(0.0f); yal1 = sc2(0.0f); ybe = sc2(1.0f);
                    }
                }
            }
        }
        Nprev = Nn;
        Hy0 = h0; Hy1 = h1; Hy2 = h2;
    }
    for (int s = 16; s > 0; s >>= 1) nclamp += __shfl_xor_sync(0xffffffffu, nclamp, s);
    if (lane == 0 && nclamp) atomicAdd(&D.ctl->clamps, nclamp);
    if (blk == 0 && threadIdx.x == 0) {
        Ctl *ct = D.ctl;
        ct->dtm2 = ct->dtm1;
        ct->dtm1 = cf.dt;
        ct->last_dt = cf.dt;
        ct->t = cf.t1;
        ct->n = cf.n + 1;
        ct->rate_bits = 0ull;
    }
}

// two blocks of 4 warps per multiprocessor (up to 255 registers a thread)
template <int YS, bool FRIC = false>
__global__ void __launch_bounds__(128, 2) k_rhs_sw2(Dev<float> D, int nstrip, int rows)
{
    rhs_sw2_body<YS, FRIC>(D, blockIdx.x, nstrip, rows);
}

// ------------------------------------------------------------------ y-line solves

// Three launches instead of one block scan: (A) every (column, chunk of KY
// rows) summarises its chunk -- the forward elimination y_j = m_j r_j + e_j y_{j-1}
// as y_end = A y_in + B, and the back substitution x_j = y_j - c'_j x_{j+1} as
// x_first = al0 + al1 y_in + be x_after (y is affine in y_in); (B) one warp per
// column scans the summaries (forward, then backward); (C) every chunk
// recomputes its y from y_in, substitutes back from x_after, and updates Q.
// No thread waits on another inside a kernel; all accesses are coalesced
// across 32 columns.
template <typename T, int KY>
__device__ __forceinline__ void ysum_body(const Dev<T> &D, int bx, int by, int nch, T *sums)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    const int i = bx * 32 + threadIdx.x;
    const int k = by * blockDim.y + threadIdx.y;
    const int nx = D.nx, ny = D.ny;
    if (i >= nx || k >= nch) return;
    const int j0 = k * KY;
    T yt = (T)0, Pi = (T)1, al0 = (T)0, al1 = (T)0, be = (T)1;
    T rr[KY], mm[KY], ee[KY], cc[KY];
#pragma unroll
    for (int q = 0; q < KY; q++) {
        const int j = j0 + q;
        const bool v = j < ny;
        const long long o = v ? fidx(D, i, j) : 0;
        T r = v ? D.dV[o] : (T)0;
        if (j == 0) r += D.corrS[i];
        if (j == ny - 1) r += D.corrN[i];
        rr[q] = r;
        mm[q] = v ? D.fym[o] : (T)0;
        ee[q] = v ? D.fye[o] : (T)1;
        cc[q] = v ? D.fyc[o] : (T)0;
    }
#pragma unroll
    for (int q = 0; q < KY; q++) {
        yt = mm[q] * rr[q] + ee[q] * yt;
        Pi = ee[q] * Pi;
        al0 = al0 + be * yt;
        al1 = al1 + be * Pi;
        be = -cc[q] * be;
    }
    const int ns = ychunk_stride(nch);
    const long long s = (long long)nx * ns, o = (long long)i * ns + k;
    sums[o] = Pi;            // A
    sums[s + o] = yt;        // B
    sums[2 * s + o] = al0;
    sums[3 * s + o] = al1;
    sums[4 * s + o] = be;
}

template <typename T, int KY>
__global__ void __launch_bounds__(256) k_ysum(Dev<T> D, int nch, T *sums)
{
    ysum_body<T, KY>(D, blockIdx.x, blockIdx.y, nch, sums);
}

// A column of more than 32 CPL chunks: the warp passes over segments of 32 CPL
// chunks, forward with the carried y, then backward with the carried x; the
// y entering each chunk goes to yin on the forward pass and is read back by
// the same lane on the backward pass.  sums, yin, xaft point at the column.
template <typename T, int CPL>
__device__ __noinline__ void yscan_long(int nch, const T *sums, long long s, T *yin, T *xaft, int lane)
{
    const int nseg = (nch + 32 * CPL - 1) / (32 * CPL);
    T carry = (T)0;
    for (int g = 0; g < nseg; g++) {
        const int c0 = g * 32 * CPL + lane * CPL;
        T a_[CPL], b_[CPL];
#pragma unroll
        for (int q = 0; q < CPL; q++) {
            const bool v = c0 + q < nch;
            a_[q] = v ? sums[c0 + q] : (T)1;
            b_[q] = v ? sums[s + c0 + q] : (T)0;
        }
        T A = (T)1, B = (T)0;
#pragma unroll
        for (int q = 0; q < CPL; q++) { B = a_[q] * B + b_[q]; A = a_[q] * A; }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T Ap = __shfl_up_sync(0xffffffffu, A, o), Bp = __shfl_up_sync(0xffffffffu, B, o);
            if (lane >= o) { B = A * Bp + B; A = A * Ap; }
        }
        T Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
        if (lane == 0) { Ae = (T)1; Be = (T)0; }
        T y = Ae * carry + Be;
#pragma unroll
        for (int q = 0; q < CPL; q++) {
            if (c0 + q < nch) yin[c0 + q] = y;
            y = a_[q] * y + b_[q];
        }
        carry = __shfl_sync(0xffffffffu, y, 31);
    }
    carry = (T)0;
    for (int g = nseg - 1; g >= 0; g--) {
        const int c0 = g * 32 * CPL + lane * CPL;
        T a_[CPL], b_[CPL];
#pragma unroll
        for (int q = 0; q < CPL; q++) {
            const bool v = c0 + q < nch;
            a_[q] = v ? sums[2 * s + c0 + q] + sums[3 * s + c0 + q] * yin[c0 + q] : (T)0;
            b_[q] = v ? sums[4 * s + c0 + q] : (T)1;
        }
        T al = (T)0, bb = (T)1;
#pragma unroll
        for (int q = CPL - 1; q >= 0; q--) { al = a_[q] + b_[q] * al; bb = b_[q] * bb; }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T ap = __shfl_down_sync(0xffffffffu, al, o), bp = __shfl_down_sync(0xffffffffu, bb, o);
            if (lane + o < 32) { al = al + bb * ap; bb = bb * bp; }
        }
        T an = __shfl_down_sync(0xffffffffu, al, 1), bn = __shfl_down_sync(0xffffffffu, bb, 1);
        if (lane == 31) { an = (T)0; bn = (T)1; }
        T x = an + bn * carry;
#pragma unroll
        for (int q = CPL - 1; q >= 0; q--) {
            if (c0 + q < nch) xaft[c0 + q] = x;
            x = a_[q] + b_[q] * x;
        }
        carry = __shfl_sync(0xffffffffu, x, 0);
    }
}

template <typename T>
__device__ __forceinline__ void yscan_body(const Dev<T> &D, int blk, int nch, const T *sums, T *yin, T *xaft)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    const int i = (int)((blk * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int nx = D.nx;
    if (i >= nx) return;
    const int ns = ychunk_stride(nch);
    const long long s = (long long)nx * ns, base = (long long)i * ns;
    constexpr int CPL = 8;  // chunks per lane: 256 chunks per pass of the warp
    if (nch > 32 * CPL) {
        yscan_long<T, CPL>(nch, sums + base, s, yin + base, xaft + base, lane);
        return;
    }
    // all five summaries of the lane's chunks are loaded up front, as vectors
    // (the per-column stride is a multiple of 8 chunks); chunks past nch are
    // replaced by identities
    T a_[CPL], b_[CPL], s2[CPL], s3[CPL], s4[CPL];
    const bool any = lane * CPL < nch;
    if (any) {
        const T *p = sums + base + lane * CPL;
        vload_k<T, CPL>(p, a_);
        vload_k<T, CPL>(p + s, b_);
        vload_k<T, CPL>(p + 2 * s, s2);
        vload_k<T, CPL>(p + 3 * s, s3);
        vload_k<T, CPL>(p + 4 * s, s4);
    }
#pragma unroll
    for (int q = 0; q < CPL; q++) {
        if (lane * CPL + q >= nch) { a_[q] = (T)1; b_[q] = (T)0; s2[q] = (T)0; s3[q] = (T)0; s4[q] = (T)1; }
    }
    // forward: lane composes its chunks, warp scan, exclusive values per chunk
    T A = (T)1, B = (T)0;
#pragma unroll
    for (int q = 0; q < CPL; q++) {
        B = a_[q] * B + b_[q];
        A = a_[q] * A;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T Ap = __shfl_up_sync(0xffffffffu, A, o), Bp = __shfl_up_sync(0xffffffffu, B, o);
        if (lane >= o) { B = A * Bp + B; A = A * Ap; }
    }
    T y = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0) y = (T)0;
    T yk[CPL];
#pragma unroll
    for (int q = 0; q < CPL; q++) {
        yk[q] = y;
        y = a_[q] * y + b_[q];
    }
    // backward: x_first(k) = (al0 + al1 y_in(k)) + be x_after(k)
    T al = (T)0, bb = (T)1;
#pragma unroll
    for (int q = 0; q < CPL; q++) {
        a_[q] = s2[q] + s3[q] * yk[q];
        b_[q] = s4[q];
    }
#pragma unroll
    for (int q = CPL - 1; q >= 0; q--) { al = a_[q] + b_[q] * al; bb = b_[q] * bb; }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T ap = __shfl_down_sync(0xffffffffu, al, o), bp = __shfl_down_sync(0xffffffffu, bb, o);
        if (lane + o < 32) { al = al + bb * ap; bb = bb * bp; }
    }
    T x = __shfl_down_sync(0xffffffffu, al, 1);
    if (lane == 31) x = (T)0;
    T xk[CPL];
#pragma unroll
    for (int q = CPL - 1; q >= 0; q--) {
        xk[q] = x;
        x = a_[q] + b_[q] * x;
    }
    if (any) {
        vstore_k<T, CPL>(yin + base + lane * CPL, yk);
        vstore_k<T, CPL>(xaft + base + lane * CPL, xk);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_yscan(Dev<T> D, int nch, const T *sums, T *yin, T *xaft)
{
    yscan_body<T>(D, blockIdx.x, nch, sums, yin, xaft);
}

template <typename T, int KY>
__device__ __forceinline__ void yapply_body(const Dev<T> &D, int bx, int by, int nch, const T *yin, const T *xaft)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    const int i = bx * blockDim.x + threadIdx.x;
    const int k = by * blockDim.y + threadIdx.y;
    const int nx = D.nx, ny = D.ny;
    if (i >= nx || k >= nch) return;
    const int j0 = k * KY;
    const long long bo = (long long)i * ychunk_stride(nch) + k;
    // all loads of a phase are issued before any store, so they overlap
    T rr[KY], mm[KY], ee[KY];
#pragma unroll
    for (int q = 0; q < KY; q++) {
        const int j = j0 + q;
        const bool v = j < ny;
        const long long o = v ? fidx(D, i, j) : 0;
        T r = v ? D.dV[o] : (T)0;
        if (j == 0) r += D.corrS[i];
        if (j == ny - 1) r += D.corrN[i];
        rr[q] = r;
        mm[q] = v ? D.fym[o] : (T)0;
        ee[q] = v ? D.fye[o] : (T)1;
    }
    T y = yin[bo];
#pragma unroll
    for (int q = 0; q < KY; q++) { y = mm[q] * rr[q] + ee[q] * y; rr[q] = y; }
    T cc[KY], Qo[KY], cq[KY];
#pragma unroll
    for (int q = 0; q < KY; q++) {
        const int j = j0 + q;
        const bool v = j < ny;
        const long long o = v ? fidx(D, i, j) : 0;
        cc[q] = v ? D.fyc[o] : (T)0;
        Qo[q] = v ? D.Q[o] : (T)0;
        cq[q] = (v && D.kahan) ? D.cQ[o] : (T)0;
    }
    T x = xaft[bo];
    const T gxi = D.gx[i];
#pragma unroll
    for (int q = KY - 1; q >= 0; q--) {
        x = rr[q] - cc[q] * x;
        T Qn, cn = (T)0;
        if (D.kahan) {
            T yy = x - cq[q];
            Qn = Qo[q] + yy;
            cn = (Qn - Qo[q]) - yy;
        } else {
            Qn = Qo[q] + x;
        }
        const int j = j0 + q;
        const T gyq = D.gy[min(j, ny - 1)];
        if (tlt(gxi, (T)1) || tlt(gyq, (T)1)) {  // the product of factors in [0, 1] is below 1
            const T gm = gxi * gyq;
            Qn *= gm;
            cn *= gm;
        }
        Qo[q] = Qn;
        cq[q] = cn;
    }
#pragma unroll
    for (int q = 0; q < KY; q++) {
        const int j = j0 + q;
        if (j < ny) {
            const long long o = fidx(D, i, j);
            D.Q[o] = Qo[q];
            if (D.kahan) D.cQ[o] = cq[q];
        }
    }
}

template <typename T, int KY>
__global__ void __launch_bounds__(256) k_yapply(Dev<T> D, int nch, const T *yin, const T *xaft)
{
    yapply_body<T, KY>(D, blockIdx.x, blockIdx.y, nch, yin, xaft);
}
// double precision: three blocks per multiprocessor (at most 85 registers)
template <int KY>
__global__ void __launch_bounds__(256, 3) k_yapply_d(Dev<double> D, int nch, const double *yin, const double *xaft)
{
    yapply_body<double, KY>(D, blockIdx.x, blockIdx.y, nch, yin, xaft);
}

// ------------------------------------------------------------------ x-line solves

// vload_k when pred, zeros otherwise (no memory access)
template <typename T, int K>
__device__ __forceinline__ void vload_k_if(bool pred, const T *p, T *out)
{
    if (pred) {
        vload_k<T, K>(p, out);
    } else {
#pragma unroll
        for (int q = 0; q < K; q++) out[q] = (T)0;
    }
}
template <typename T, int K>
__device__ __forceinline__ void load_halo_chunk_if(bool pred, const T *row, int ib, int lane, T *v)
{
    vload_k_if<T, K>(pred, row + ib, v + 1);
    T left = __shfl_up_sync(0xffffffffu, v[K], 1);
    T right = __shfl_down_sync(0xffffffffu, v[1], 1);
    if (lane == 0) left = row[ib - 1];
    if (lane == 31 && pred) right = row[ib + K];
    v[0] = left;
    v[K + 1] = right;
}

// One CTA per x-line (Eq. 19).  Thread t owns the K contiguous elements
// [K t, K t + K) in registers.  Forward elimination y_i = m_i r_i + e_i y_{i-1}
// and back substitution x_i = y_i - c'_i x_{i+1} are affine recurrences: each
// thread composes its chunk, a block scan (warp shuffles, then across warps in
// shared memory) gives the value entering each chunk, and the chunk is
// finished in registers.  Also: F* at the new level from Q^{n+1} on the
// right-hand side (sequential cross form), compensated P update, sponge on w
// and P, and the Eq. 22 rate of the finished state (one atomic per block).
template <typename T, int K>
// (double precision, 4 elements a thread: two rows per multiprocessor at 64
// registers, so one row's barrier waits overlap the other's FP64 work)
__global__ void __launch_bounds__(512, (sizeof(T) == 8 && K == 4) ? 2 : 1) k_xsolve(Dev<T> D, double forced_dt_next)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    __shared__ T sA[32], sB[32];
    __shared__ double smax[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    const int j = blockIdx.x;
    const int nx = D.nx;
    const int ib = t * K;
    const long long rowo = fidx(D, 0, j);
    const bool seq = D.cross_mode != 0;

    T r[K], m[K], e[K];
    vload_k<T, K>(D.dU + rowo + ib, r);
    vload_k<T, K>(D.fxm + rowo + ib, m);
    vload_k<T, K>(D.fxe + rowo + ib, e);
    if (seq && sizeof(T) == 8) {
        // F* of Eq. 14 at the new level from Q^{n+1} (ghosts at t_{n+1}),
        // with the coefficients formed at set-up
        const T half_rdx = (T)0.5 * D.rdx, half_rdy = (T)0.5 * D.rdy, q_rdxy = (T)0.25 * D.rdx * D.rdy;
        T c1[K], c2[K], c3[K];
        vload_k<T, K>(D.fsc1 + rowo + ib, c1);
        vload_k<T, K>(D.fsc2 + rowo + ib, c2);
        vload_k<T, K>(D.fsc3 + rowo + ib, c3);
        T q0[K + 2], qm[K + 2], qp[K + 2];
        load_halo_chunk<T, K>(D.Q + rowo, ib, lane, q0);
        load_halo_chunk<T, K>(D.Q + rowo - D.pitch, ib, lane, qm);
        load_halo_chunk<T, K>(D.Q + rowo + D.pitch, ib, lane, qp);
#pragma unroll
        for (int q = 0; q < K; q++) {
            T Q_x = (q0[q + 2] - q0[q]) * half_rdx;
            T Q_y = (qp[q + 1] - qm[q + 1]) * half_rdy;
            T Q_xy = (qp[q + 2] - qm[q + 2] - qp[q] + qm[q]) * q_rdxy;
            r[q] += c1[q] * Q_y + c2[q] * Q_x + c3[q] * Q_xy;
        }
    } else if (seq) {
        // F* of Eq. 14 at the new level from Q^{n+1} (ghosts at t_{n+1})
        const T half_rdx = (T)0.5 * D.rdx, half_rdy = (T)0.5 * D.rdy, q_rdxy = (T)0.25 * D.rdx * D.rdy;
        const T kB = D.Bd + (T)1 / (T)3, sixth = (T)1 / (T)6;
        T dd[K + 2], ddy[K];
        {
            T b0[K + 2], bm[K + 2], bp[K + 2];
            load_halo_chunk<T, K>(D.bC + rowo, ib, lane, b0);
            load_halo_chunk<T, K>(D.bC + rowo - D.pitch, ib, lane, bm);
            load_halo_chunk<T, K>(D.bC + rowo + D.pitch, ib, lane, bp);
#pragma unroll
            for (int q = 0; q < K + 2; q++) dd[q] = tmax(D.w_s - b0[q], (T)0);
#pragma unroll
            for (int q = 0; q < K; q++)
                ddy[q] = (tmax(D.w_s - bp[q + 1], (T)0) - tmax(D.w_s - bm[q + 1], (T)0)) * half_rdy;
        }
        T q0[K + 2], qm[K + 2], qp[K + 2];
        load_halo_chunk<T, K>(D.Q + rowo, ib, lane, q0);
        load_halo_chunk<T, K>(D.Q + rowo - D.pitch, ib, lane, qm);
        load_halo_chunk<T, K>(D.Q + rowo + D.pitch, ib, lane, qp);
#pragma unroll
        for (int q = 0; q < K; q++) {
            T d = dd[q + 1];
            T ddx = (dd[q + 2] - dd[q]) * half_rdx;
            T Q_x = (q0[q + 2] - q0[q]) * half_rdx;
            T Q_y = (qp[q + 1] - qm[q + 1]) * half_rdy;
            T Q_xy = (qp[q + 2] - qm[q + 2] - qp[q] + qm[q]) * q_rdxy;
            r[q] += d * ddx * Q_y * sixth + d * ddy[q] * Q_x * sixth + kB * d * d * Q_xy;
        }
    }
    const T corrW = D.corrW[j], corrE = D.corrE[j];
#pragma unroll
    for (int q = 0; q < K; q++) {
        int i = ib + q;
        if (i == 0) r[q] += corrW;
        if (i == nx - 1) r[q] += corrE;
        if (i >= nx) { r[q] = (T)0; m[q] = (T)0; e[q] = (T)1; }
    }
    // ---- forward elimination: compose, block scan (earlier chunks first)
    T A = (T)1, B = (T)0;
#pragma unroll
    for (int q = 0; q < K; q++) { B = m[q] * r[q] + e[q] * B; A = e[q] * A; }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T Ap = __shfl_up_sync(0xffffffffu, A, o);
        T Bp = __shfl_up_sync(0xffffffffu, B, o);
        if (lane >= o) { B = A * Bp + B; A = A * Ap; }
    }
    if (lane == 31) { sA[wid] = A; sB[wid] = B; }
    T Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0) { Ae = (T)1; Be = (T)0; }
    __syncthreads();
    if (wid == 0) {
        T a = lane < nw ? sA[lane] : (T)1, b = lane < nw ? sB[lane] : (T)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T ap = __shfl_up_sync(0xffffffffu, a, o);
            T bp = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) { b = a * bp + b; a = a * ap; }
        }
        T bx = __shfl_up_sync(0xffffffffu, b, 1);
        if (lane == 0) bx = (T)0;
        if (lane < nw) sB[lane] = bx;  // y entering warp `lane`
    }
    __syncthreads();
    T y = Ae * sB[wid] + Be;
#pragma unroll
    for (int q = 0; q < K; q++) { y = m[q] * r[q] + e[q] * y; r[q] = (ib + q < nx) ? y : (T)0; }
    __syncthreads();  // sA/sB reused below

    // ---- back substitution: compose from the end, block suffix scan
    T c[K];
    vload_k<T, K>(D.fxc + rowo + ib, c);
#pragma unroll
    for (int q = 0; q < K; q++)
        if (ib + q >= nx) c[q] = (T)0;
    T al = (T)0, be = (T)1;
#pragma unroll
    for (int q = K - 1; q >= 0; q--) { al = r[q] - c[q] * al; be = -c[q] * be; }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T ap = __shfl_down_sync(0xffffffffu, al, o);
        T bp = __shfl_down_sync(0xffffffffu, be, o);
        if (lane + o < 32) { al = al + be * ap; be = be * bp; }
    }
    if (lane == 0) { sA[wid] = al; sB[wid] = be; }
    T an = __shfl_down_sync(0xffffffffu, al, 1), bn = __shfl_down_sync(0xffffffffu, be, 1);
    if (lane == 31) { an = (T)0; bn = (T)1; }
    __syncthreads();
    if (wid == 0) {
        T a = lane < nw ? sA[lane] : (T)0, b = lane < nw ? sB[lane] : (T)1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T ap = __shfl_down_sync(0xffffffffu, a, o);
            T bp = __shfl_down_sync(0xffffffffu, b, o);
            if (lane + o < 32) { a = a + b * ap; b = b * bp; }
        }
        T ax = __shfl_down_sync(0xffffffffu, a, 1);
        if (lane == 31) ax = (T)0;
        if (lane < nw) sA[lane] = ax;  // x just after warp `lane`
    }
    __syncthreads();
    T x = an + bn * sA[wid];
#pragma unroll
    for (int q = K - 1; q >= 0; q--) { x = r[q] - c[q] * x; r[q] = x; }

    // ---- P^{n+1} = P^n + x (compensated), sponge on w and P, Eq. 22 rate
    T *Pr = D.P + rowo, *cPr = D.cP + rowo;
    T *wr = D.w[cf.wc ^ 1] + rowo, *cwr = D.cw + rowo;
    T Pv[K], cPv[K], wv[K], Qv[K], bv[K];
    vload_k<T, K>(Pr + ib, Pv);
    if (D.kahan) vload_k<T, K>(cPr + ib, cPv);
    vload_k<T, K>(wr + ib, wv);
    vload_k<T, K>(D.Q + rowo + ib, Qv);
    vload_k<T, K>(D.bC + rowo + ib, bv);
    const T gyj = D.gy[j];
    T mu = (T)0, mv = (T)0;  // largest |u| + c and |v| + c (Eq. 22), scaled once
    bool bad = false;
#pragma unroll
    for (int q = 0; q < K; q++) {
        const int i = ib + q;
        if (i >= nx) continue;
        T Pn, cn = (T)0;
        if (D.kahan) {
            T yy = r[q] - cPv[q];
            Pn = Pv[q] + yy;
            cn = (Pn - Pv[q]) - yy;
        } else {
            Pn = Pv[q] + r[q];
        }
        T wq = wv[q];
        const T gxi = D.gx[i];
        if (tlt(gxi, (T)1) || tlt(gyj, (T)1)) {  // the product of factors in [0, 1] is below 1
            const T gm = gxi * gyj;
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
        const IvC<T> ic = ivc(h, D.g, tsqrt(D.g), D.eps, D.hdry);
        T u = ic.iv * Pn, v = ic.iv * Qv[q];
        T cc = ic.c;
        mu = tmax(mu, fabs(u) + cc);
        mv = tmax(mv, fabs(v) + cc);
        if (!tfinite(wq) || !tfinite(Pn) || !tfinite(Qv[q])) bad = true;
    }
    vstore_k<T, K>(Pr + ib, Pv);
    if (D.kahan) vstore_k<T, K>(cPr + ib, cPv);

    double rr = (double)tmax(mu * D.rdx, mv * D.rdy);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rr = fmax(rr, __shfl_xor_sync(0xffffffffu, rr, o));
    bool anybad = __any_sync(0xffffffffu, bad);
    if (lane == 0) smax[wid] = anybad ? -1.0 : rr;
    __syncthreads();
    if (t == 0) {
        double mx = 0.0;
        bool fl = false;
        for (int q = 0; q < nw; q++) {
            if (smax[q] < 0.0) fl = true;
            else mx = fmax(mx, smax[q]);
        }
        if (fl) atomicOr(&D.ctl->err, ERR_NONFINITE);
        atomicMax(&D.ctl->rate_bits, dbits(mx));
        next_step_controller(D, forced_dt_next, gridDim.x);
    }
}

// ------------------------------------------------------------------ x-line solves, TMA-staged

// Shared-memory address of a generic pointer (for PTX operands).
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// 1D bulk copy global -> shared, completion counted on the mbarrier (TMA)
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity`; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, long long limit)
{
    for (long long it = 0; it < limit; it++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Staging of the persistent x-solver: the row's input arrays dU, m, e, c', P,
// cP, w (interior span) and Q, bC at rows j-1, j, j+1 (interior span plus one
// 16-byte halo on each side) in shared memory.
constexpr int XT_ARR_PLAIN = 7, XT_ARR_HALO = 6;

// Issue the bulk copies of row j into one staging buffer (thread 0).
template <typename T>
__device__ __forceinline__ void xrow_issue(const Dev<T> &D, const Coef &cf, int j, T *S, int span,
                                           unsigned long long *bar)
{
    const int hx = D.hx, hspan = span + 2 * hx;
    const long long rowo = fidx(D, 0, j);
    const bool seq = D.cross_mode != 0;
    const unsigned pb = (unsigned)(span * sizeof(T)), hb = (unsigned)(hspan * sizeof(T));
    unsigned total = 6u * pb + (D.kahan ? pb : 0u) + 2u * hb + (seq ? 4u * hb : 0u);
    mbar_expect_tx(bar, total);
    tma_load_1d(S + 0 * span, D.dU + rowo, pb, bar);
    tma_load_1d(S + 1 * span, D.fxm + rowo, pb, bar);
    tma_load_1d(S + 2 * span, D.fxe + rowo, pb, bar);
    tma_load_1d(S + 3 * span, D.fxc + rowo, pb, bar);
    tma_load_1d(S + 4 * span, D.P + rowo, pb, bar);
    if (D.kahan) tma_load_1d(S + 5 * span, D.cP + rowo, pb, bar);
    tma_load_1d(S + 6 * span, D.w[cf.wc ^ 1] + rowo, pb, bar);
    T *sH = S + 7 * span;
    const T *Qr = D.Q + rowo - hx, *br = D.bC + rowo - hx;
    tma_load_1d(sH + 0 * hspan, Qr, hb, bar);
    tma_load_1d(sH + 3 * hspan, br, hb, bar);
    if (seq) {
        tma_load_1d(sH + 1 * hspan, Qr - D.pitch, hb, bar);
        tma_load_1d(sH + 2 * hspan, Qr + D.pitch, hb, bar);
        tma_load_1d(sH + 4 * hspan, br - D.pitch, hb, bar);
        tma_load_1d(sH + 5 * hspan, br + D.pitch, hb, bar);
    }
}

// Persistent x-line solver: one block per SM walks rows blockIdx.x,
// blockIdx.x + gridDim.x, ...; two staging buffers, so the bulk copies of the
// next row are in flight while the current row is solved (same arithmetic as
// k_xsolve).
template <typename T, int K>
__global__ void __launch_bounds__(512, 1) k_xsolve_pipe(Dev<T> D, int span, double forced_dt_next)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ T sA[32], sB[32], sC[32], sD[32];
    __shared__ double smax[32];
    const int hx = D.hx;
    const int hspan = span + 2 * hx;
    const size_t per = (size_t)7 * span + (size_t)6 * hspan;
    T *buf0 = reinterpret_cast<T *>(smem_raw), *buf1 = buf0 + per;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    const int nx = D.nx, ny = D.ny;
    const bool seq = D.cross_mode != 0;
    const int ib = t * K;
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
        if ((int)blockIdx.x < ny) xrow_issue(D, cf, blockIdx.x, buf0, span, &bar[0]);
    }
    __syncthreads();
    T mu = (T)0, mv = (T)0;  // largest |u| + c and |v| + c (Eq. 22), scaled once
    bool bad = false, failed = false;
    int it = 0;
    for (int j = blockIdx.x; j < ny; j += gridDim.x, it++) {
        T *S = (it & 1) ? buf1 : buf0;
        unsigned long long *b = &bar[it & 1];
        const bool ok = mbar_wait_bounded(b, (unsigned)((it >> 1) & 1), 1LL << 24);
        if (__syncthreads_or(!ok)) { failed = true; break; }
        // the other buffer was released by the barrier that ended the last row;
        // order those shared-memory reads before the bulk copies overwrite it
        if (t == 0 && j + (int)gridDim.x < ny) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            xrow_issue(D, cf, j + gridDim.x, (it & 1) ? buf0 : buf1, span, &bar[(it + 1) & 1]);
        }
        const long long rowo = fidx(D, 0, j);
        T *sdU = S, *sm = S + span, *se = S + 2 * span, *sc = S + 3 * span, *sP = S + 4 * span;
        T *scP = S + 5 * span, *sw = S + 6 * span, *sH = S + 7 * span;
        T r[K], m[K], e[K];
        vload_k<T, K>(sdU + ib, r);
        vload_k<T, K>(sm + ib, m);
        vload_k<T, K>(se + ib, e);
        T Qc[K + 2], bc_[K + 2];
        load_halo_chunk<T, K>(sH + 0 * hspan + hx, ib, lane, Qc);
        load_halo_chunk<T, K>(sH + 3 * hspan + hx, ib, lane, bc_);
        if (seq) {
            const T half_rdx = (T)0.5 * D.rdx, half_rdy = (T)0.5 * D.rdy, q_rdxy = (T)0.25 * D.rdx * D.rdy;
            const T kB = D.Bd + (T)1 / (T)3, sixth = (T)1 / (T)6;
            T qm[K + 2], qp[K + 2], bm[K], bp[K];
            load_halo_chunk<T, K>(sH + 1 * hspan + hx, ib, lane, qm);
            load_halo_chunk<T, K>(sH + 2 * hspan + hx, ib, lane, qp);
            vload_k<T, K>(sH + 4 * hspan + hx + ib, bm);
            vload_k<T, K>(sH + 5 * hspan + hx + ib, bp);
            // ghosts of Q^{n+1} at t_{n+1}: columns -1 and nx (W/E rule) in rows
            // j-1, j, j+1 inside the domain, then the whole ghost row (S/N rule)
            // when row j-1 or j+1 lies outside; each thread fixes what it reads
            if (ib == 0) {
                if (j - 1 >= 0) qm[0] = D.bc[SW] == MAKER ? D.mqW[j - 1] : qm[1];
                Qc[0] = D.bc[SW] == MAKER ? D.mqW[j] : Qc[1];
                if (j + 1 < ny) qp[0] = D.bc[SW] == MAKER ? D.mqW[j + 1] : qp[1];
            }
            if (nx - 1 >= ib && nx - 1 < ib + K) {
                const int qe = nx - ib;  // index of column nx in the halo arrays
#pragma unroll
                for (int q = 1; q <= K; q++)
                    if (q == qe) {
                        if (j - 1 >= 0) qm[q + 1] = D.bc[SE] == MAKER ? D.mqE[j - 1] : qm[q];
                        Qc[q + 1] = D.bc[SE] == MAKER ? D.mqE[j] : Qc[q];
                        if (j + 1 < ny) qp[q + 1] = D.bc[SE] == MAKER ? D.mqE[j + 1] : qp[q];
                    }
            }
            if (j == 0 || j == ny - 1) {
                const int side = j == 0 ? SS : SN;
                const T *mq = side == SS ? D.mqS : D.mqN;  // maker Q at columns -1..nx
#pragma unroll
                for (int q = 0; q < K + 2; q++) {
                    const int c = ib - 1 + q;
                    const T gv = D.bc[side] == MAKER ? mq[min(max(c, -1), nx) + 1] : -Qc[q];
                    if (j == 0) qm[q] = gv;  // (no pointer select: keeps both arrays in registers)
                    else qp[q] = gv;
                }
            }
#pragma unroll
            for (int q = 0; q < K; q++) {
                T d = tmax(D.w_s - bc_[q + 1], (T)0);
                T ddx = (tmax(D.w_s - bc_[q + 2], (T)0) - tmax(D.w_s - bc_[q], (T)0)) * half_rdx;
                T ddy = (tmax(D.w_s - bp[q], (T)0) - tmax(D.w_s - bm[q], (T)0)) * half_rdy;
                T Q_x = (Qc[q + 2] - Qc[q]) * half_rdx;
                T Q_y = (qp[q + 1] - qm[q + 1]) * half_rdy;
                T Q_xy = (qp[q + 2] - qm[q + 2] - qp[q] + qm[q]) * q_rdxy;
                r[q] += d * ddx * Q_y * sixth + d * ddy * Q_x * sixth + kB * d * d * Q_xy;
            }
        }
        const T corrW = D.corrW[j], corrE = D.corrE[j];
#pragma unroll
        for (int q = 0; q < K; q++) {
            int i = ib + q;
            if (i == 0) r[q] += corrW;
            if (i == nx - 1) r[q] += corrE;
            if (i >= nx) { r[q] = (T)0; m[q] = (T)0; e[q] = (T)1; }
        }
        T A = (T)1, B = (T)0;
#pragma unroll
        for (int q = 0; q < K; q++) { B = m[q] * r[q] + e[q] * B; A = e[q] * A; }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T Ap = __shfl_up_sync(0xffffffffu, A, o);
            T Bp = __shfl_up_sync(0xffffffffu, B, o);
            if (lane >= o) { B = A * Bp + B; A = A * Ap; }
        }
        if (lane == 31) { sA[wid] = A; sB[wid] = B; }
        T Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
        if (lane == 0) { Ae = (T)1; Be = (T)0; }
        __syncthreads();
        // y entering this warp: the totals of the warps before it, applied in order to y = 0
        T yw = (T)0;
        for (int q = 0; q < wid; q++) yw = sA[q] * yw + sB[q];
        T y = Ae * yw + Be;
#pragma unroll
        for (int q = 0; q < K; q++) { y = m[q] * r[q] + e[q] * y; r[q] = (ib + q < nx) ? y : (T)0; }
        T c[K];
        vload_k<T, K>(sc + ib, c);
#pragma unroll
        for (int q = 0; q < K; q++)
            if (ib + q >= nx) c[q] = (T)0;
        T al = (T)0, be = (T)1;
#pragma unroll
        for (int q = K - 1; q >= 0; q--) { al = r[q] - c[q] * al; be = -c[q] * be; }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T ap = __shfl_down_sync(0xffffffffu, al, o);
            T bp = __shfl_down_sync(0xffffffffu, be, o);
            if (lane + o < 32) { al = al + be * ap; be = be * bp; }
        }
        if (lane == 0) { sC[wid] = al; sD[wid] = be; }
        T an = __shfl_down_sync(0xffffffffu, al, 1), bn = __shfl_down_sync(0xffffffffu, be, 1);
        if (lane == 31) { an = (T)0; bn = (T)1; }
        __syncthreads();
        // x just after this warp: the totals of the warps after it, from the end
        T xw = (T)0;
        for (int q = nw - 1; q > wid; q--) xw = sC[q] + sD[q] * xw;
        T x = an + bn * xw;
#pragma unroll
        for (int q = K - 1; q >= 0; q--) { x = r[q] - c[q] * x; r[q] = x; }

        T *Pr = D.P + rowo, *cPr = D.cP + rowo, *cwr = D.cw + rowo;
        T *wrow = D.w[cf.wc ^ 1] + rowo;
        T Pv[K], cPv[K], wv[K];
        const T *Qv = Qc + 1, *bv = bc_ + 1;
        vload_k<T, K>(sP + ib, Pv);
        if (D.kahan) vload_k<T, K>(scP + ib, cPv);
        vload_k<T, K>(sw + ib, wv);
        const T gyj = D.gy[j];
#pragma unroll
        for (int q = 0; q < K; q++) {
            const int i = ib + q;
            if (i >= nx) continue;
            T Pn, cn = (T)0;
            if (D.kahan) {
                T yy = r[q] - cPv[q];
                Pn = Pv[q] + yy;
                cn = (Pn - Pv[q]) - yy;
            } else {
                Pn = Pv[q] + r[q];
            }
            T wq = wv[q];
            const T gxi = D.gx[i];
            if (tlt(gxi, (T)1) || tlt(gyj, (T)1)) {  // the product of factors in [0, 1] is below 1
                const T gm = gxi * gyj;
                T h = tmax(wq - bv[q], (T)0), d = tmax(D.w_s - bv[q], (T)0);
                wq = bv[q] + (d + gm * (h - d));
                wrow[i] = wq;
                if (D.kahan) cwr[i] = (T)0;
                Pn *= gm;
                cn *= gm;
            }
            Pv[q] = Pn;
            cPv[q] = cn;
            T h = tmax(wq - bv[q], (T)0);
            const IvC<T> ic = ivc(h, D.g, tsqrt(D.g), D.eps, D.hdry);
            T u = ic.iv * Pn, v = ic.iv * Qv[q];
            T cc = ic.c;
            mu = tmax(mu, fabs(u) + cc);
            mv = tmax(mv, fabs(v) + cc);
            if (!tfinite(wq) || !tfinite(Pn) || !tfinite(Qv[q])) bad = true;
        }
        if (ib < nx) {
            vstore_k<T, K>(Pr + ib, Pv);
            if (D.kahan) vstore_k<T, K>(cPr + ib, cPv);
        }
        // the wait barrier at the top of the next iteration also releases this buffer
    }
    if (failed) {
        // copies did not complete: flag it, wait (bounded) for what is in
        // flight, let the controller of the next step stop the run
        mbar_wait_bounded(&bar[0], 0, 1LL << 22);
        mbar_wait_bounded(&bar[1], 0, 1LL << 22);
        if (t == 0) {
            atomicOr(&D.ctl->err, ERR_DEVICE_WAIT);
            next_step_controller(D, 0.0, gridDim.x);
        }
        return;
    }
    double rr = (double)tmax(mu * D.rdx, mv * D.rdy);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rr = fmax(rr, __shfl_xor_sync(0xffffffffu, rr, o));
    bool anybad = __any_sync(0xffffffffu, bad);
    if (lane == 0) smax[wid] = anybad ? -1.0 : rr;
    __syncthreads();
    if (t == 0) {
        double mx = 0.0;
        bool fl = false;
        for (int q = 0; q < nw; q++) {
            if (smax[q] < 0.0) fl = true;
            else mx = fmax(mx, smax[q]);
        }
        if (fl) atomicOr(&D.ctl->err, ERR_NONFINITE);
        atomicMax(&D.ctl->rate_bits, dbits(mx));
        next_step_controller(D, forced_dt_next, gridDim.x);
    }
}

// ---- one warp per x-line
//
// A warp solves row j in chunks of 32 K elements (lane l owns the K
// contiguous elements c0 + l K ...).  Forward elimination runs over the chunks
// left to right: local composition, a warp scan of the affine maps and the
// carry y entering the chunk; the y values go to the warp's shared-memory
// row.  Back substitution runs right to left with the carry x after the chunk
// and finishes each chunk at once: compensated P update, sponge on w and P,
// Eq. 22 rate.  Warps never wait on each other, so every row of the grid can
// be in flight at once.  Same arithmetic as k_xsolve.
// FIXED: the default configuration (sequential cross form, compensated
// accumulation) compiled in, no run-time switches on either
template <typename T, int K, bool FIXED = false>
__device__ __forceinline__ void xsolve_row_warp(const Dev<T> &D, const Coef &cf, int j, T *ys, T &rate, bool &bad)
{
    const int lane = threadIdx.x & 31;
    // largest |u| + c and |v| + c of Eq. 22 over the lane's cells, scaled once at the
    // end (scaling by a positive constant keeps the order, so the largest rate)
    T mu = (T)0, mv = (T)0;
    const int nx = D.nx, ny = D.ny;
    const bool seq = FIXED || D.cross_mode != 0;
    const bool kah = FIXED || D.kahan != 0;
    const long long rowo = fidx(D, 0, j);
    const T *Qr = D.Q + rowo, *br = D.bC + rowo;
    const T corrW = D.corrW[j], corrE = D.corrE[j];
    const T half_rdx = (T)0.5 * D.rdx, half_rdy = (T)0.5 * D.rdy, q_rdxy = (T)0.25 * D.rdx * D.rdy;
    const T kB = D.Bd + (T)1 / (T)3, sixth = (T)1 / (T)6;
    T carry = (T)0;
    int c0 = 0;
    for (; c0 < nx; c0 += 32 * K) {
        const int ib = c0 + lane * K;
        // lanes past the row end load nothing; the lane holding column nx still
        // loads (its first element is the right neighbour of the last cell)
        const bool act = ib <= nx;
        T r[K], m[K], e[K];
        vload_k_if<T, K>(act, D.dU + rowo + ib, r);
        vload_k_if<T, K>(act, D.fxm + rowo + ib, m);
        vload_k_if<T, K>(act, D.fxe + rowo + ib, e);
        if (seq) {
            // double precision: the F* coefficients formed at set-up;
            // single precision: the still depth from the bed rows
            constexpr bool F64 = sizeof(T) == 8;
            T Qc[K + 2], bc_[F64 ? 1 : K + 2], qm[K + 2], qp[K + 2], bm[F64 ? 1 : K], bp[F64 ? 1 : K];
            T c1[F64 ? K : 1], c2[F64 ? K : 1], c3[F64 ? K : 1];
            load_halo_chunk_if<T, K>(act, Qr, ib, lane, Qc);
            load_halo_chunk_if<T, K>(act, Qr - D.pitch, ib, lane, qm);
            load_halo_chunk_if<T, K>(act, Qr + D.pitch, ib, lane, qp);
            if constexpr (F64) {
                vload_k_if<T, K>(act, D.fsc1 + rowo + ib, c1);
                vload_k_if<T, K>(act, D.fsc2 + rowo + ib, c2);
                vload_k_if<T, K>(act, D.fsc3 + rowo + ib, c3);
            } else {
                load_halo_chunk_if<T, K>(act, br, ib, lane, bc_);
                vload_k_if<T, K>(act, br - D.pitch + ib, bm);
                vload_k_if<T, K>(act, br + D.pitch + ib, bp);
            }
            // ghosts of Q^{n+1} at t_{n+1}, as in k_xsolve_pipe
            if (ib == 0) {
                if (j - 1 >= 0) qm[0] = D.bc[SW] == MAKER ? D.mqW[j - 1] : qm[1];
                Qc[0] = D.bc[SW] == MAKER ? D.mqW[j] : Qc[1];
                if (j + 1 < ny) qp[0] = D.bc[SW] == MAKER ? D.mqW[j + 1] : qp[1];
            }
            if (nx - 1 >= ib && nx - 1 < ib + K) {
                const int qe = nx - ib;
#pragma unroll
                for (int q = 1; q <= K; q++)
                    if (q == qe) {
                        if (j - 1 >= 0) qm[q + 1] = D.bc[SE] == MAKER ? D.mqE[j - 1] : qm[q];
                        Qc[q + 1] = D.bc[SE] == MAKER ? D.mqE[j] : Qc[q];
                        if (j + 1 < ny) qp[q + 1] = D.bc[SE] == MAKER ? D.mqE[j + 1] : qp[q];
                    }
            }
            if (j == 0 || j == ny - 1) {
                const int side = j == 0 ? SS : SN;
                const T *mq = side == SS ? D.mqS : D.mqN;
#pragma unroll
                for (int q = 0; q < K + 2; q++) {
                    const int cc = ib - 1 + q;
                    const T gv = D.bc[side] == MAKER ? mq[min(max(cc, -1), nx) + 1] : -Qc[q];
                    if (j == 0) qm[q] = gv;
                    else qp[q] = gv;
                }
            }
#pragma unroll
            for (int q = 0; q < K; q++) {
                T Q_x = (Qc[q + 2] - Qc[q]) * half_rdx;
                T Q_y = (qp[q + 1] - qm[q + 1]) * half_rdy;
                T Q_xy = (qp[q + 2] - qm[q + 2] - qp[q] + qm[q]) * q_rdxy;
                if constexpr (F64) {
                    r[q] += c1[q] * Q_y + c2[q] * Q_x + c3[q] * Q_xy;
                } else {
                    T d = tmax(D.w_s - bc_[q + 1], (T)0);
                    T ddx = (tmax(D.w_s - bc_[q + 2], (T)0) - tmax(D.w_s - bc_[q], (T)0)) * half_rdx;
                    T ddy = (tmax(D.w_s - bp[q], (T)0) - tmax(D.w_s - bm[q], (T)0)) * half_rdy;
                    r[q] += d * ddx * Q_y * sixth + d * ddy * Q_x * sixth + kB * d * d * Q_xy;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < K; q++) {
            const int i = ib + q;
            if (i == 0) r[q] += corrW;
            if (i == nx - 1) r[q] += corrE;
            if (i >= nx) { r[q] = (T)0; m[q] = (T)0; e[q] = (T)1; }
        }
        T A = (T)1, B = (T)0;
#pragma unroll
        for (int q = 0; q < K; q++) { B = m[q] * r[q] + e[q] * B; A = e[q] * A; }
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
        for (int q = 0; q < K; q++) { y = m[q] * r[q] + e[q] * y; r[q] = y; }
        vstore_k<T, K>(ys + ib, r);
        carry = __shfl_sync(0xffffffffu, y, 31);
    }
    __syncwarp();
    // back substitution, last chunk first
    carry = (T)0;
    const T gyj = D.gy[j];
    T *Pr = D.P + rowo, *cPr = D.cP + rowo, *cwr = D.cw + rowo;
    T *wrow = D.w[cf.wc ^ 1] + rowo;
    for (c0 -= 32 * K; c0 >= 0; c0 -= 32 * K) {
        const int ib = c0 + lane * K;
        const bool act = ib < nx;
        T x[K], c[K], Pv[K], cPv[K], wv[K], Qv[K], bv[K], gxv[K];
        vload_k<T, K>(ys + ib, x);
        vload_k_if<T, K>(act, D.gx + ib, gxv);
        vload_k_if<T, K>(act, D.fxc + rowo + ib, c);
        vload_k_if<T, K>(act, Pr + ib, Pv);
        vload_k_if<T, K>(act && kah, cPr + ib, cPv);
        vload_k_if<T, K>(act, wrow + ib, wv);
        vload_k_if<T, K>(act, Qr + ib, Qv);
        vload_k_if<T, K>(act, br + ib, bv);
#pragma unroll
        for (int q = 0; q < K; q++)
            if (ib + q >= nx) { c[q] = (T)0; x[q] = (T)0; }
        T al = (T)0, be = (T)1;
#pragma unroll
        for (int q = K - 1; q >= 0; q--) { al = x[q] - c[q] * al; be = -c[q] * be; }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T ap = __shfl_down_sync(0xffffffffu, al, o);
            T bp = __shfl_down_sync(0xffffffffu, be, o);
            if (lane + o < 32) { al = al + be * ap; be = be * bp; }
        }
        T an = __shfl_down_sync(0xffffffffu, al, 1), bn = __shfl_down_sync(0xffffffffu, be, 1);
        if (lane == 31) { an = (T)0; bn = (T)1; }
        T xx = an + bn * carry;
#pragma unroll
        for (int q = K - 1; q >= 0; q--) { xx = x[q] - c[q] * xx; x[q] = xx; }
        carry = __shfl_sync(0xffffffffu, xx, 0);
#pragma unroll
        for (int q = 0; q < K; q++) {
            const int i = ib + q;
            if (i >= nx) continue;
            T Pn, cn = (T)0;
            if (kah) {
                T yy = x[q] - cPv[q];
                Pn = Pv[q] + yy;
                cn = (Pn - Pv[q]) - yy;
            } else {
                Pn = Pv[q] + x[q];
            }
            T wq = wv[q];
            if (tlt(gxv[q], (T)1) || tlt(gyj, (T)1)) {  // the product of factors in [0, 1] is below 1
                const T gm = gxv[q] * gyj;
                T h = tmax(wq - bv[q], (T)0), d = tmax(D.w_s - bv[q], (T)0);
                wq = bv[q] + (d + gm * (h - d));
                wrow[i] = wq;
                if (kah) cwr[i] = (T)0;
                Pn *= gm;
                cn *= gm;
            }
            Pv[q] = Pn;
            cPv[q] = cn;
            T h = tmax(wq - bv[q], (T)0);
            const IvC<T> ic = ivc(h, D.g, tsqrt(D.g), D.eps, D.hdry);
            T u = ic.iv * Pn, v = ic.iv * Qv[q];
            T cc = ic.c;
            mu = tmax(mu, fabs(u) + cc);
            mv = tmax(mv, fabs(v) + cc);
            if (!tfinite(wq) || !tfinite(Pn) || !tfinite(Qv[q])) bad = true;
        }
        if (ib < nx) {
            vstore_k<T, K>(Pr + ib, Pv);
            if (kah) vstore_k<T, K>(cPr + ib, cPv);
        }
    }
    rate = tmax(rate, tmax(mu * D.rdx, mv * D.rdy));
}

constexpr int XW_WARPS = 4;  // rows (warps) per block of the batched warp-per-row x-solvers
// rows (warps) per block of the single-domain warp-per-row x-solver: small
// blocks spread the rows evenly over the multiprocessors (2048 rows: 12 or 14
// on each of 152, where blocks of four rows left some with 16)
constexpr int XW_ONE = 2;

// shared memory of the warp-per-row x-solver: one y row per warp
template <typename T, int K>
static size_t xwarp_smem(int nx, int nw = XW_WARPS)
{
    const int span = 32 * K;
    return (size_t)nw * (size_t)((nx + span - 1) / span) * span * sizeof(T);
}

// rows blk * NW + warp of one domain; the controller of the domain's next
// step runs in the last of its nparts blocks
template <typename T, int K, bool FIXED = false, int NW = XW_WARPS>
__device__ __forceinline__ void xsolve_warp_body(const Dev<T> &D, int blk, unsigned nparts, int yrow,
                                                 double forced_dt_next)
{
    const Coef cf = *D.coef;
    if (!cf.active) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double smax[NW];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *ys = reinterpret_cast<T *>(smem_raw) + (size_t)wid * yrow;
    const int j = blk * NW + wid;
    T rate = (T)0;
    bool bad = false;
    if (j < D.ny) xsolve_row_warp<T, K, FIXED>(D, cf, j, ys, rate, bad);
    double rr = (double)rate;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rr = fmax(rr, __shfl_xor_sync(0xffffffffu, rr, o));
    const bool anybad = __any_sync(0xffffffffu, bad);
    if (lane == 0) smax[wid] = anybad ? -1.0 : rr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        bool fl = false;
        for (int q = 0; q < NW; q++) {
            if (smax[q] < 0.0) fl = true;
            else mx = fmax(mx, smax[q]);
        }
        if (fl) atomicOr(&D.ctl->err, ERR_NONFINITE);
        atomicMax(&D.ctl->rate_bits, dbits(mx));
        next_step_controller(D, forced_dt_next, nparts);
    }
}

template <typename T, int K, bool FIXED = false>
__global__ void __launch_bounds__(32 * XW_ONE, (sizeof(T) == 4 ? 16 : 8) / XW_ONE) k_xsolve_warp(Dev<T> D, int yrow, double forced_dt_next)
{
    xsolve_warp_body<T, K, FIXED, XW_ONE>(D, blockIdx.x, gridDim.x, yrow, forced_dt_next);
}

// shared memory bytes of the TMA x-solver for a row span
template <typename T>
static size_t xtma_smem(int span, int hx)
{
    return ((size_t)XT_ARR_PLAIN * span + (size_t)XT_ARR_HALO * (span + 2 * hx)) * sizeof(T);
}

// ------------------------------------------------------------------ set-up of a new domain
//
// The static geometry, the line factors and the initial state of a domain,
// computed on the device in FP64 from device copies of the caller's arrays
// (KP07 corner bed, Sec. 3; Eq. 21 coefficients; h = max(d + eta0, 0)).
// bed at the (nx+5) x (ny+5) corners -2..nx+2, mirrored past the edges
template <typename T>
__global__ void k_setup_corner(Dev<T> D, SetupArgs A)
{
    const int cx = D.nx + 5, cy = D.ny + 5;
    const long long n = (long long)cx * cy;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % cx) - 2, j = (int)(q / cx) - 2;
        const int is = i < 0 ? -i : (i > D.nx ? 2 * D.nx - i : i);
        const int js = j < 0 ? -j : (j > D.ny ? 2 * D.ny - j : j);
        D.corner[q] = (T)A.bed[(size_t)is + (size_t)js * (D.nx + 1)];
    }
}

// bed at the centres (mean of the 4 face values) and still depth, cells -2..nx+1 x -2..ny+1
template <typename T>
__global__ void k_setup_centres(Dev<T> D, SetupArgs A)
{
    const int w = D.nx + 4, h = D.ny + 4;
    const long long n = (long long)w * h;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % w) - 2, j = (int)(q / w) - 2;
        auto K = [&](int a, int b) {
            const int is = a < 0 ? -a : (a > D.nx ? 2 * D.nx - a : a);
            const int js = b < 0 ? -b : (b > D.ny ? 2 * D.ny - b : b);
            return A.bed[(size_t)is + (size_t)js * (D.nx + 1)];
        };
        const double bw = 0.5 * (K(i, j) + K(i, j + 1)), be = 0.5 * (K(i + 1, j) + K(i + 1, j + 1));
        const double bs = 0.5 * (K(i, j) + K(i + 1, j)), bn = 0.5 * (K(i, j + 1) + K(i + 1, j + 1));
        const double b = 0.25 * (bw + be + bs + bn);
        const long long c = fidx(D, i, j);
        A.bCd[c] = b;
        A.dd[c] = fmax(A.w_s - b, 0.0);
        if constexpr (sizeof(T) == 4) {
            // single precision: from the FP32 corners with the RHS kernels' own
            // rounding, so every kernel sees bitwise the same still depth
            const T *kc = D.corner;
            const int cp = D.cpitch;
            auto KF = [&](int a, int bb) { return kc[(long long)(bb + 2) * cp + (a + 2)]; };
            D.bC[c] = bed_centre(KF(i, j), KF(i + 1, j), KF(i, j + 1), KF(i + 1, j + 1));
        } else {
            D.bC[c] = (T)b;
        }
    }
}

// Double precision: the F*, G* coefficients of Eqs. 14-15 at the interior
// cell centres from the still depth d and its central differences d_x, d_y
// (as the step kernels form them): F* = c1 Q_y + c2 Q_x + c3 Q_xy and
// G* = c2 P_x + c1 P_y + c3 P_xy with c1 = d d_x / 6, c2 = d d_y / 6,
// c3 = (B + 1/3) d^2.  At GB300's FP64 rate a load is cheaper than the dozen
// operations that form them in every step.
template <typename T>
__global__ void k_setup_fstar(Dev<T> D)
{
    const int nx = D.nx;
    const long long n = (long long)nx * D.ny;
    const T half_rdx = (T)0.5 * D.rdx, half_rdy = (T)0.5 * D.rdy;
    const T kB = D.Bd + (T)1 / (T)3, sixth = (T)1 / (T)6;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx), j = (int)(q / nx);
        auto dep = [&](int a, int b) { return tmax(D.w_s - D.bC[fidx(D, a, b)], (T)0); };
        const T d = dep(i, j);
        const T ddx = (dep(i + 1, j) - dep(i - 1, j)) * half_rdx;
        const T ddy = (dep(i, j + 1) - dep(i, j - 1)) * half_rdy;
        const long long c = fidx(D, i, j);
        D.fsc1[c] = d * ddx * sixth;
        D.fsc2[c] = d * ddy * sixth;
        D.fsc3[c] = kB * d * d;
        // the RHS kernel's other static terms, in its order of operations
        const T *kc = D.corner;
        const int cp = D.cpitch;
        auto K = [&](int a, int b) { return kc[(long long)(b + 2) * cp + (a + 2)]; };
        const T bxW = (T)0.5 * (K(i, j) + K(i, j + 1)), bxE = (T)0.5 * (K(i + 1, j) + K(i + 1, j + 1));
        const T bS = (T)0.5 * (K(i, j) + K(i + 1, j)), bN = (T)0.5 * (K(i, j + 1) + K(i + 1, j + 1));
        const T g = D.g, Bg = D.Bd * g;
        T *st = D.stat + c;
        const long long ss = D.stat_stride;
        st[ST_SX * ss] = -g * (bxE - bxW) * D.rdx;
        st[ST_MX * ss] = (T)0.5 * (bxE + bxW);
        st[ST_SY * ss] = -g * (bN - bS) * D.rdy;
        st[ST_MY * ss] = (T)0.5 * (bN + bS);
        const T bd2 = Bg * d * d;
        st[ST_BD2 * ss] = bd2;
        st[ST_BD3 * ss] = bd2 * d;
        st[ST_DDX * ss] = ddx;
        st[ST_DDY * ss] = ddy;
    }
}

// Thomas factors (m, -a m, c' = c m) of every x-line and y-line, boundary
// rows closed: wall or sponge = odd mirror of the normal flux (the outside
// coefficient moves onto the diagonal), maker = the outside value is known
// (its coefficient goes to cW..cN).  The rows of Eq. 21 come from the still
// depth with reciprocals of the cell size taken once.
//
// The pivots p_k = b_k - a_k c_{k-1} / p_{k-1} (m_k = 1 / p_k) are ratios
// p_k = u_k / u_{k-1} of the linear recurrence u_k = b_k u_{k-1} - a_k c_{k-1}
// u_{k-2} (u_{-1} = 1, u_{-2} = 0), whose step is the 2x2 matrix
// [[b_k, -a_k c_{k-1}], [1, 0]] acting on (u_{k-1}, u_{k-2}).  A line is cut
// into FS_SEG segments, one thread each: every thread multiplies its
// segment's matrices, the product of the segments before it gives the state
// its segment starts from, and a second walk of the segment produces the
// factors.  The recurrence carries its dominant solution, so the segments'
// rounding does not grow (about 1e-14 relative against 1e-15 for one walk
// along the line); states and products are rescaled by exact powers of two.
// A block holds 32 lines (lanes) x FS_SEG segments (warps), x-lines in blocks
// 0 .. ceil(ny/32)-1 and y-lines after them; the still depth is loaded FS_CH
// cells ahead, and an x-line warp writes its rows through shared memory,
// FS_CH consecutive values of a row at a time.
constexpr int FS_SEG = 8, FS_CH = 8;

template <typename T>
static size_t setup_factors_smem()
{
    return (size_t)FS_SEG * 32 * 4 * sizeof(double) + (size_t)FS_SEG * 3 * FS_CH * 33 * sizeof(T);
}

__device__ __forceinline__ double pow2_inv_scale(double x)
{
    return x == 0.0 ? 1.0 : scalbn(1.0, -ilogb(x));
}

template <typename T>
__global__ void __launch_bounds__(32 * FS_SEG) k_setup_factors(Dev<T> D, SetupArgs A)
{
    extern __shared__ __align__(16) unsigned char fs_smem[];
    double *Gs = reinterpret_cast<double *>(fs_smem);  // [FS_SEG][32][4]
    T *tile = reinterpret_cast<T *>(fs_smem + (size_t)FS_SEG * 32 * 4 * sizeof(double)) +
              (size_t)(threadIdx.x >> 5) * 3 * FS_CH * 33;  // this warp's [3][FS_CH][33]
    const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const double kB = A.Bd + 1.0 / 3.0;
    const int nx = D.nx, ny = D.ny;
    const int nbx = (ny + 31) / 32;
    const bool xline = (int)blockIdx.x < nbx;
    const int line0 = (xline ? (int)blockIdx.x : (int)blockIdx.x - nbx) * 32;
    const int line = line0 + lane;
    const int nlines = xline ? ny : nx;
    if (line0 >= nlines) return;  // (block-uniform)
    const bool valid = line < nlines;
    const int n = xline ? nx : ny;
    const int S = (n + FS_SEG - 1) / FS_SEG;
    const int kb = min(n, seg * S), ke = min(n, kb + S);
    const double h = xline ? A.dx : A.dy;
    const double r2h = 0.5 / h, r6h = 1.0 / (6.0 * h), rh2 = 1.0 / (h * h);
    const int lo = xline ? A.bt[0] : A.bt[2], hi = xline ? A.bt[1] : A.bt[3];
    double *cfirst = xline ? A.cW : A.cS, *clast = xline ? A.cE : A.cN;
    T *fm = xline ? D.fxm : D.fym, *fe = xline ? D.fxe : D.fye, *fc = xline ? D.fxc : D.fyc;
    auto at = [&](int k, int l) { return xline ? fidx(D, k, l) : fidx(D, l, k); };
    auto dd = [&](int k) { return valid ? A.dd[at(k, line)] : 1.0; };
    // row k of the line from the still depth at k-1, k, k+1, ends closed;
    // `outside` receives the coefficient of the outside neighbour at an end
    auto row = [&](int k, double dm, double d0, double dp, double &a, double &b, double &c, double &outside) {
        const double gd = (dp - dm) * r2h;
        const double t1 = d0 * gd * r6h, t2 = kB * d0 * d0 * rh2;
        a = t1 - t2;
        b = 1.0 + 2.0 * t2;
        c = -t1 - t2;
        if (k == 0) { outside = a; if (lo != MAKER) b -= a; a = 0.0; }
        if (k == n - 1) { outside = c; if (hi != MAKER) b -= c; c = 0.0; }
    };
    // c of the row before the segment (a_kb multiplies it)
    double cprev0 = 0.0;
    if (kb > 0 && kb < n) {
        double a, b, c, o;
        row(kb - 1, dd(kb - 2), dd(kb - 1), dd(kb), a, b, c, o);
        cprev0 = c;
    }

    // ---- pass 1: product of the segment's step matrices
    double g00 = 1.0, g01 = 0.0, g10 = 0.0, g11 = 1.0;
    {
        double dm = kb < n ? dd(kb - 1) : 1.0, d0 = kb < n ? dd(kb) : 1.0, cprev = cprev0;
        for (int k0 = kb; k0 < ke; k0 += FS_CH) {
            double dn[FS_CH];
#pragma unroll
            for (int q = 0; q < FS_CH; q++) dn[q] = k0 + q < ke ? dd(k0 + q + 1) : 1.0;
#pragma unroll
            for (int q = 0; q < FS_CH; q++) {
                const int k = k0 + q;
                if (k >= ke) break;
                double a, b, c, o;
                row(k, dm, d0, dn[q], a, b, c, o);
                const double qa = a * cprev;
                const double n00 = b * g00 - qa * g10, n01 = b * g01 - qa * g11;
                g10 = g00;
                g11 = g01;
                g00 = n00;
                g01 = n01;
                cprev = c;
                dm = d0;
                d0 = dn[q];
            }
            const double sc = pow2_inv_scale(fmax(fmax(fabs(g00), fabs(g01)), fmax(fabs(g10), fabs(g11))));
            g00 *= sc; g01 *= sc; g10 *= sc; g11 *= sc;
        }
    }
    double *gme = Gs + ((size_t)seg * 32 + lane) * 4;
    gme[0] = g00; gme[1] = g01; gme[2] = g10; gme[3] = g11;
    __syncthreads();
    // state (u_{kb-1}, u_{kb-2}) from the products of the segments before
    double u = 1.0, v = 0.0;
    for (int s2 = 0; s2 < seg; s2++) {
        const double *gp = Gs + ((size_t)s2 * 32 + lane) * 4;
        const double nu = gp[0] * u + gp[1] * v, nv = gp[2] * u + gp[3] * v;
        const double sc = pow2_inv_scale(fmax(fabs(nu), fabs(nv)));
        u = nu * sc;
        v = nv * sc;
    }

    // ---- pass 2: the factors
    double dm = kb < n ? dd(kb - 1) : 1.0, d0 = kb < n ? dd(kb) : 1.0, cprev = cprev0;
    for (int k0 = kb; k0 < ke; k0 += FS_CH) {
        double dn[FS_CH];
#pragma unroll
        for (int q = 0; q < FS_CH; q++) dn[q] = k0 + q < ke ? dd(k0 + q + 1) : 1.0;
#pragma unroll
        for (int q = 0; q < FS_CH; q++) {
            const int k = k0 + q;
            if (k >= ke) break;
            double a, b, c, o = 0.0;
            row(k, dm, d0, dn[q], a, b, c, o);
            if (valid) {
                if (k == 0) cfirst[line] = o;
                if (k == n - 1) clast[line] = o;
                if (!(fabs(b) > fabs(a) + fabs(c))) atomicOr(A.bad, 1u);
            }
            const double un = fma(b, u, -(a * cprev) * v);  // u_k
            const double m = u / un;                          // 1 / p_k
            v = u;
            u = un;
            cprev = c;
            dm = d0;
            d0 = dn[q];
            if (xline) {
                tile[(0 * FS_CH + q) * 33 + lane] = (T)m;
                tile[(1 * FS_CH + q) * 33 + lane] = (T)(-a * m);
                tile[(2 * FS_CH + q) * 33 + lane] = (T)(c * m);
            } else if (valid) {
                const long long o = at(k, line);
                fm[o] = (T)m;
                fe[o] = (T)(-a * m);
                fc[o] = (T)(c * m);
            }
        }
        const double sc = pow2_inv_scale(u);
        u *= sc;
        v *= sc;
        if (xline) {
            __syncwarp();
            for (int idx = lane; idx < 32 * FS_CH; idx += 32) {
                const int rr = idx / FS_CH, q = idx - rr * FS_CH, k = k0 + q;
                if (k < ke && line0 + rr < ny) {
                    const long long o = at(k, line0 + rr);
                    fm[o] = tile[(0 * FS_CH + q) * 33 + rr];
                    fe[o] = tile[(1 * FS_CH + q) * 33 + rr];
                    fc[o] = tile[(2 * FS_CH + q) * 33 + rr];
                }
            }
            __syncwarp();
        }
    }
}

// factor fields outside the interior hold the identity row (m = 0, -a m = 1, c' = 0)
template <typename T>
__global__ void k_setup_fill(Dev<T> D)
{
    const long long n = (long long)D.pitch * (D.ny + 4);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        D.fxe[q] = (T)1;
        D.fye[q] = (T)1;
    }
}

// initial state: w = b + max(d + eta0, 0), P0, Q0 (zeros where not given)
template <typename T>
__global__ void k_setup_state(Dev<T> D, SetupArgs A)
{
    const long long n = (long long)D.nx * D.ny;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k % D.nx), j = (int)(k / D.nx);
        const long long c = fidx(D, i, j);
        const double h = fmax(A.dd[c] + (A.eta0 ? A.eta0[k] : 0.0), 0.0);
        D.w[0][c] = (T)(A.bCd[c] + h);
        D.P[c] = (T)(A.P0 ? A.P0[k] : 0.0);
        D.Q[c] = (T)(A.Q0 ? A.Q0[k] : 0.0);
    }
}

template <typename T>
cudaError_t launch_setup(const Dev<T> &D, cudaStream_t st, const SetupArgs &A)
{
    const int gs = 1024;
    k_setup_fill<T><<<gs, 256, 0, st>>>(D);
    k_setup_corner<T><<<gs, 256, 0, st>>>(D, A);
    k_setup_centres<T><<<gs, 256, 0, st>>>(D, A);
    const size_t fsm = setup_factors_smem<T>();
    cudaError_t e = cudaFuncSetAttribute(k_setup_factors<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    if (e != cudaSuccess) return e;
    k_setup_factors<T><<<(D.ny + 31) / 32 + (D.nx + 31) / 32, 32 * FS_SEG, fsm, st>>>(D, A);
    if constexpr (sizeof(T) == 8) k_setup_fstar<T><<<gs, 256, 0, st>>>(D);
    k_setup_state<T><<<gs, 256, 0, st>>>(D, A);
    return cudaGetLastError();
}

// Table of the single-precision maker: cos and sin of kx x + ky y + phi of
// every component at every maker point of the maker sides (FP64, rounded to
// FP32); one thread per (component, point).
__global__ void k_setup_mtab(Dev<float> D)
{
    const int nx = D.nx, ny = D.ny, ly = ny + 4, lx = nx + 4, np = D.mpts;
    const long long n = (long long)np * D.ncomp;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(q / np), pt = (int)(q - (long long)k * np);
        int side, r;
        if (pt < 2 * ly) { side = SW; r = pt; }
        else if (pt < 4 * ly) { side = SE; r = pt - 2 * ly; }
        else if (pt < 4 * ly + 2 * lx) { side = SS; r = pt - 4 * ly; }
        else { side = SN; r = pt - 4 * ly - 2 * lx; }
        if (D.bc[side] != MAKER) continue;
        const int len = side == SW || side == SE ? ly : lx;
        const int g = r / len + 1, m = r - (g - 1) * len - 2;
        int i, j;
        if (side == SW) { i = -g; j = m; }
        else if (side == SE) { i = nx - 1 + g; j = m; }
        else if (side == SS) { i = m; j = -g; }
        else { i = m; j = ny - 1 + g; }
        const double ph = D.kx[k] * (((double)i + 0.5) * D.dxd) + D.ky[k] * (((double)j + 0.5) * D.dyd) + D.ph[k];
        double sn, cs;
        sincos(ph, &sn, &cs);
        D.mtab[q] = make_float2((float)cs, (float)sn);
    }
}

template <typename T>
cudaError_t launch_maker_table(const Dev<T> &D, cudaStream_t st)
{
    if constexpr (sizeof(T) == 4) {
        if (D.mtab && D.ncomp > 0) {
            const long long n = (long long)D.mpts * D.ncomp;
            const int blocks = (int)(n / 256 + 1 < 4096 ? n / 256 + 1 : 4096);
            k_setup_mtab<<<blocks, 256, 0, st>>>(D);
        }
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ utilities

// FP64 fused multiply-add throughput: each thread runs 8 independent chains
// x <- x a + b of n steps (|a| < 1 keeps the values bounded) and stores their
// sum, which keeps every chain live.
__global__ void __launch_bounds__(256) k_fma64(double *out, int n, double a, double b)
{
    double x[8];
#pragma unroll
    for (int q = 0; q < 8; q++) x[q] = (double)(threadIdx.x + q) * 1e-3;
    for (int i = 0; i < n; i++) {
#pragma unroll
        for (int q = 0; q < 8; q++) x[q] = fma(x[q], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; q++) s += x[q];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_fma64(double *out, int blocks, int n, cudaStream_t st)
{
    k_fma64<<<blocks, 256, 0, st>>>(out, n, 0.999, 1e-3);
    return cudaGetLastError();
}

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
        const IvC<T> ic = ivc(h, D.g, tsqrt(D.g), D.eps, D.hdry);
        T u = ic.iv * D.P[c], v = ic.iv * D.Q[c];
        T cc = ic.c;
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

// Interior field into a compact nx*ny array of O (T, or double for reads
// that widen on the device).
template <typename T, typename O>
__global__ void __launch_bounds__(256) k_extract(Dev<T> D, int wc, int field, O *out)
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
        out[q] = (O)v;
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

// ------------------------------------------------------------------ launchers

template <typename T>
static int ysplit_rows(int tune)
{
    return tune > 0 ? tune : 8;
}

template <typename T>
int ysplit_chunks(int ny, int tune)
{
    const int KY = ysplit_rows<T>(tune);
    return (ny + KY - 1) / KY;
}

template <typename T>
int step_shape_ok(int nx, int ny)
{
    // x-solver: at most 512 threads of 32 elements a row; y-solver: any
    // number of chunks (the chunk scan loops over segments of 256 chunks)
    (void)ny;
    return nx <= 512 * 32;
}

// x-solver chunk: elements per thread (a multiple of the vector width), at
// most 512 threads per row; by default 8 in single precision (two rows of
// up to 2048 cells in flight per block), 4 in double precision
template <typename T>
int x_chunk(int nx, int tune)
{
    int K = tune > 0 ? tune : (sizeof(T) == 4 ? 8 : 4);
    if (K < VecT<T>::N) K = VecT<T>::N;
    while (K < 32 && (nx + K - 1) / K > 512) K *= 2;
    return K;
}

template <typename T>
int row_pitch(int nx, int tune)
{
    int span = 32 * x_chunk<T>(nx, tune);
    return ((nx + span - 1) / span) * span + span;
}

constexpr size_t XPIPE_MAX_SMEM = 220 * 1024;

template <typename T>
cudaError_t configure(int nx)
{
    (void)nx;
    const int pb = (int)XPIPE_MAX_SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_xsolve_pipe<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, pb);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_xsolve_pipe<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, pb);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_xsolve_pipe<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, pb);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_xsolve_pipe<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, pb);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_xsolve_warp<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_xsolve_warp<T, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_xsolve_warp<T, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_xsolve_warp<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    return e;
}

// two-columns-per-lane RHS (single precision, default configuration)
static bool launch_rhs2(const Dev<float> &D, cudaStream_t st, int rows, int ky)
{
    const int nstrip = (D.nx + SW2_COLS - 1) / SW2_COLS;
    const int nband = (D.ny + rows - 1) / rows;
    const int blocks = (int)(((long long)nstrip * nband + 3) / 4);
    if (D.friction != 0.0f) {
        if (ky == 16) k_rhs_sw2<16, true><<<blocks, 128, 0, st>>>(D, nstrip, rows);
        else if (ky == 8) k_rhs_sw2<8, true><<<blocks, 128, 0, st>>>(D, nstrip, rows);
        else k_rhs_sw2<0, true><<<blocks, 128, 0, st>>>(D, nstrip, rows);
    } else if (ky == 16) k_rhs_sw2<16><<<blocks, 128, 0, st>>>(D, nstrip, rows);
    else if (ky == 8) k_rhs_sw2<8><<<blocks, 128, 0, st>>>(D, nstrip, rows);
    else k_rhs_sw2<0><<<blocks, 128, 0, st>>>(D, nstrip, rows);
    return true;
}
static bool launch_rhs2(const Dev<double> &, cudaStream_t, int, int) { return false; }

// x-solver variants (tune_xtma): 0 automatic -- in single precision the
// warp-per-row kernel where its shared-memory rows fit, else the persistent
// kernel with two staged rows where they fit, else registers only; in double
// precision the persistent kernel where it fits, else registers only;
// 1 registers only; 3 the persistent kernel where it fits; 4 the
// warp-per-row kernel where it fits.
template <typename T>
static bool xsolver_pipe_allowed(const Dev<T> &D)
{
    return D.tune_xtma == 0 || D.tune_xtma == 3;
}
// the warp-per-row x-solver (tune_xtma 4), K = 4 or 8, y row in shared memory
template <typename T>
static bool xsolver_warp(const Dev<T> &D, int nx)
{
    const int K = x_chunk<T>(nx, D.tune_xk);
    const bool want = D.tune_xtma == 4 || (D.tune_xtma == 0 && sizeof(T) == 4);
    return want && (K == 4 || K == 8) && (K == 4 ? xwarp_smem<T, 4>(nx) : xwarp_smem<T, 8>(nx)) <= 96 * 1024;
}

// the sliding-window RHS kernel's compile-time default configuration
template <typename T>
static bool rhs_fast(const Dev<T> &D)
{
    return D.theta == (T)1 && D.cross_mode != 0 && D.friction == (T)0 && (D.kahan != 0) == (sizeof(T) == 4) &&
           D.fstride * 15 < 0x7fffffffLL;
}
// the paired single-precision RHS kernel: the fast configuration, with or
// without bottom friction (tune_rows 16 asks for the one-column kernel)
template <typename T>
static bool rhs_pair(const Dev<T> &D)
{
    return sizeof(T) == 4 && D.tune_rhs1 == 0 && D.tune_rows != 16 && D.theta == (T)1 &&
           D.cross_mode != 0 && D.kahan != 0 && D.fstride * 15 < 0x7fffffffLL;
}
// Rows per warp of the sliding-window RHS kernels.  A warp walks its strip's
// rows plus 4 halo rows, and two blocks of four warps fit a multiprocessor, so
// a launch takes about waves x (rows + 4) row steps, waves = blocks / (2 x
// multiprocessors) rounded up.  Where 64-row strips fill the device (at least
// one wave: 2048 x 2048 and up) the paired kernel takes 64; on smaller grids
// the multiple of the y-chunk rows in {64, 48, 32, 24, 16} that minimises the
// estimate (24 at 1000 x 1500, 16 below a million cells).  The one-column
// kernels are compiled for 16, 32 and 64 rows (and 128 with the chunk
// summaries of 8 rows) and take 64, or 32 when 64-row strips give fewer than
// four warps per multiprocessor; in double precision 128 where 128-row strips
// still give seven warps per multiprocessor (2048 x 2048).
template <typename T>
static int rhs_rows(const Dev<T> &D)
{
    const bool pair = rhs_pair(D);
    // 128 rows: the one-column kernel that forms the chunk summaries only
    const bool r128 = !pair && rhs_fast(D) && D.tune_ysum == 0 && ysplit_rows<T>(D.tune_yk) == 8;
    if (D.tune_rows == 128) return r128 ? 128 : 64;
    if (D.tune_rows > 0) return pair || D.tune_rows == 16 || D.tune_rows == 64 ? D.tune_rows : 32;
    if (!pair) {
        const long long nstrip = (D.nx + SW_COLS - 1) / SW_COLS;
        // double precision on large grids: 128-row strips (4 halo rows in 132
        // against 4 in 68; the kernel is bound by the FP64 pipe, which two
        // warps per scheduler keep busy)
        if (sizeof(T) == 8 && r128 && nstrip * ((D.ny + 127) / 128) >= 7LL * D.nsm) return 128;
        const long long warps64 = nstrip * ((D.ny + 63) / 64);
        return warps64 >= 4LL * D.nsm ? 64 : 32;
    }
    const int ky = ysplit_rows<T>(D.tune_yk);
    const long long nstrip = (D.nx + SW2_COLS - 1) / SW2_COLS, slots = 8LL * D.nsm;
    if (nstrip * ((D.ny + 63) / 64) >= slots) return 64;
    const int cand[5] = {64, 48, 32, 24, 16};
    int best = 64;
    long long best_cost = -1;
    for (int q = 0; q < 5; q++) {
        const int r = cand[q];
        if (r % ky) continue;
        const long long warps = nstrip * ((D.ny + r - 1) / r);
        const long long cost = ((warps + slots - 1) / slots) * (r + 4);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = r; }
    }
    return best;
}
// 1 when the RHS kernel forms the y-line chunk summaries (no k_ysum launch)
template <typename T>
static bool rhs_fuses_ysum(const Dev<T> &D)
{
    const int rows = rhs_rows(D);
    const bool pair_fuses = rhs_pair(D) && rows % ysplit_rows<T>(D.tune_yk) == 0;  // bands start on chunks
    return (pair_fuses || (rhs_fast(D) && rows != 16)) && D.tune_ysum == 0;
}

// Dynamic shared memory of the ghost kernels: the single-precision maker's
// per-step factors.
template <typename T>
static int ghost_smem(const Dev<T> &D)
{
    return sizeof(T) == 4 ? maker_step_bytes(D.ncomp) : 0;
}

// One step on stream st: ghost cells, RHS + combine, y-line solves, (ghost
// cells of Q where the x-solver does not patch them itself), x-line solves
// whose last block runs the controller of the next step with forced_dt_next
// (> 0: replay that step size).  With ev != nullptr, events ev[0..5] are
// recorded before each launch and after the last (kernel timing).
template <typename T>
static cudaError_t step_impl(const Dev<T> &D, cudaStream_t st, double forced_dt_next, cudaEvent_t *ev)
{
    const int nx = D.nx, ny = D.ny;
    long long nwork = 4LL * ny + 4LL * (nx + 4) + 2LL * ny + 2LL * nx;
    int gb = (int)((nwork + 255) / 256);
    if (ev) cudaEventRecord(ev[0], st);
    if (D.ncomp <= MK_FEW) k_ghost<T, MK_FEW><<<gb, 256, ghost_smem(D), st>>>(D);
    else k_ghost<T><<<gb, 256, ghost_smem(D), st>>>(D);
    if (ev) cudaEventRecord(ev[1], st);
    const int rows = rhs_rows(D);
    const int nstrip = (nx + SW_COLS - 1) / SW_COLS;
    const int nband = (ny + rows - 1) / rows;
    const long long nwarp = (long long)nstrip * nband;
    const int blocks = (int)((nwarp + 3) / 4);
    const bool fast = rhs_fast(D);
    const bool ysum_fused = rhs_fuses_ysum(D);  // the RHS kernel forms the y-line chunk summaries
    const bool t1 = D.theta == (T)1;
    if (rhs_pair(D)) {
        launch_rhs2(D, st, rows, ysum_fused ? ysplit_rows<T>(D.tune_yk) : 0);
    } else if (fast && ysum_fused) {
        const int KY = ysplit_rows<T>(D.tune_yk);
        if (rows == 32) {
            if (KY == 16) k_rhs_sw<T, 32, true, true, 16><<<blocks, 128, 0, st>>>(D, nstrip);
            else k_rhs_sw<T, 32, true, true, 8><<<blocks, 128, 0, st>>>(D, nstrip);
        } else if (rows == 128) {
            k_rhs_sw<T, 128, true, true, 8><<<blocks, 128, 0, st>>>(D, nstrip);
        } else {
            if (KY == 16) k_rhs_sw<T, 64, true, true, 16><<<blocks, 128, 0, st>>>(D, nstrip);
            else k_rhs_sw<T, 64, true, true, 8><<<blocks, 128, 0, st>>>(D, nstrip);
        }
    } else if (fast) {
        if (rows == 16) k_rhs_sw<T, 16, true, true><<<blocks, 128, 0, st>>>(D, nstrip);
        else if (rows == 32) k_rhs_sw<T, 32, true, true><<<blocks, 128, 0, st>>>(D, nstrip);
        else k_rhs_sw<T, 64, true, true><<<blocks, 128, 0, st>>>(D, nstrip);
    } else if (rows == 16) {
        if (t1) k_rhs_sw<T, 16, true, false><<<blocks, 128, 0, st>>>(D, nstrip);
        else k_rhs_sw<T, 16, false, false><<<blocks, 128, 0, st>>>(D, nstrip);
    } else if (rows == 64) {
        if (t1) k_rhs_sw<T, 64, true, false><<<blocks, 128, 0, st>>>(D, nstrip);
        else k_rhs_sw<T, 64, false, false><<<blocks, 128, 0, st>>>(D, nstrip);
    } else {
        if (t1) k_rhs_sw<T, 32, true, false><<<blocks, 128, 0, st>>>(D, nstrip);
        else k_rhs_sw<T, 32, false, false><<<blocks, 128, 0, st>>>(D, nstrip);
    }
    if (ev) cudaEventRecord(ev[2], st);
    {
        const int KY = ysplit_rows<T>(D.tune_yk);
        const int nch = (ny + KY - 1) / KY;
        dim3 gb2((nx + 31) / 32, (nch + 7) / 8);
        if (!ysum_fused) {
            if (KY == 8) k_ysum<T, 8><<<gb2, dim3(32, 8), 0, st>>>(D, nch, D.ysums);
            else k_ysum<T, 16><<<gb2, dim3(32, 8), 0, st>>>(D, nch, D.ysums);
        }
        k_yscan<T><<<(int)(((long long)nx * 32 + 255) / 256), 256, 0, st>>>(D, nch, D.ysums, D.yin, D.yxa);
        // one chunk of 256 adjacent columns per block: each row segment a block
        // reads is 1 KB contiguous
        const dim3 gw((nx + 255) / 256, nch);
        if constexpr (sizeof(T) == 8) {
            if (KY == 8) k_yapply_d<8><<<gw, dim3(256, 1), 0, st>>>(D, nch, D.yin, D.yxa);
            else k_yapply_d<16><<<gw, dim3(256, 1), 0, st>>>(D, nch, D.yin, D.yxa);
        } else {
            if (KY == 8) k_yapply<T, 8><<<gw, dim3(256, 1), 0, st>>>(D, nch, D.yin, D.yxa);
            else k_yapply<T, 16><<<gw, dim3(256, 1), 0, st>>>(D, nch, D.yin, D.yxa);
        }
    }
    if (ev) cudaEventRecord(ev[3], st);
    const int K = x_chunk<T>(nx, D.tune_xk);
    int thr = ((nx + K - 1) / K + 31) / 32 * 32;
    const int span = thr * K;
    const size_t xs = xtma_smem<T>(span, D.hx);
    const bool xwarp = xsolver_warp(D, nx);
    const bool pipe = !xwarp && xsolver_pipe_allowed(D) && 2 * xs <= XPIPE_MAX_SMEM;
    if (D.cross_mode != 0 && !xwarp && !pipe) {
        long long ng = 4LL * ny + 4LL * (nx + 4);
        k_ghost_q<T><<<(int)((ng + 255) / 256), 256, ghost_smem(D), st>>>(D);
    }
    if (ev) cudaEventRecord(ev[4], st);
    if (xwarp) {
        const int xb = (ny + XW_ONE - 1) / XW_ONE;
        const bool fixed = D.cross_mode != 0 && D.kahan != 0;
        if (K == 4) {
            const int yrow = (nx + 127) / 128 * 128;
            if (fixed) k_xsolve_warp<T, 4, true><<<xb, 32 * XW_ONE, xwarp_smem<T, 4>(nx, XW_ONE), st>>>(D, yrow, forced_dt_next);
            else k_xsolve_warp<T, 4><<<xb, 32 * XW_ONE, xwarp_smem<T, 4>(nx, XW_ONE), st>>>(D, yrow, forced_dt_next);
        } else {
            const int yrow = (nx + 255) / 256 * 256;
            if (fixed) k_xsolve_warp<T, 8, true><<<xb, 32 * XW_ONE, xwarp_smem<T, 8>(nx, XW_ONE), st>>>(D, yrow, forced_dt_next);
            else k_xsolve_warp<T, 8><<<xb, 32 * XW_ONE, xwarp_smem<T, 8>(nx, XW_ONE), st>>>(D, yrow, forced_dt_next);
        }
    } else if (pipe) {
        const int grid = min(ny, D.nsm);
        if (K == 4) k_xsolve_pipe<T, 4><<<grid, thr, 2 * xs, st>>>(D, span, forced_dt_next);
        else if (K == 8) k_xsolve_pipe<T, 8><<<grid, thr, 2 * xs, st>>>(D, span, forced_dt_next);
        else if (K == 16) k_xsolve_pipe<T, 16><<<grid, thr, 2 * xs, st>>>(D, span, forced_dt_next);
        else k_xsolve_pipe<T, 32><<<grid, thr, 2 * xs, st>>>(D, span, forced_dt_next);
    } else if (K == 4) k_xsolve<T, 4><<<ny, thr, 0, st>>>(D, forced_dt_next);
    else if (K == 8) k_xsolve<T, 8><<<ny, thr, 0, st>>>(D, forced_dt_next);
    else if (K == 16) k_xsolve<T, 16><<<ny, thr, 0, st>>>(D, forced_dt_next);
    else k_xsolve<T, 32><<<ny, thr, 0, st>>>(D, forced_dt_next);
    if (ev) cudaEventRecord(ev[5], st);
    return cudaGetLastError();
}

// 1 when the x-solver patches the Q ghosts itself (no k_ghost_q launch)
template <typename T>
int xsolver_staged(const Dev<T> &D, int nx)
{
    const int K = x_chunk<T>(nx, D.tune_xk);
    const int thr = ((nx + K - 1) / K + 31) / 32 * 32;
    const size_t xs = xtma_smem<T>(thr * K, D.hx);
    return xsolver_warp(D, nx) || (xsolver_pipe_allowed(D) && 2 * xs <= XPIPE_MAX_SMEM);
}

// kernel launches of one step, by the decisions step_impl takes
template <typename T>
int step_launches(const Dev<T> &D)
{
    const int nx = D.nx;
    const bool ghost_q = D.cross_mode != 0 && !xsolver_staged(D, nx);
    const int ylaunch = rhs_fuses_ysum(D) ? 2 : 3;
    return 1 /* ghost */ + 1 /* rhs */ + ylaunch + (ghost_q ? 1 : 0) + 1 /* x-solver */;
}

template <typename T>
cudaError_t launch_prologue(const Dev<T> &D, cudaStream_t st, double forced_dt, double t_end, long long max_steps)
{
    k_prologue<T><<<1, 1, 0, st>>>(D, forced_dt, t_end, max_steps);
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
    k_extract<T, T><<<gb, 256, 0, st>>>(D, wc, field, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extract_f64(const Dev<T> &D, cudaStream_t st, int wc, int field, double *out)
{
    long long ncell = (long long)D.nx * D.ny;
    int gb = (int)std::min<long long>((ncell + 255) / 256, 4096);
    k_extract<T, double><<<gb, 256, 0, st>>>(D, wc, field, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mass(const Dev<T> &D, cudaStream_t st, int wc, double *partial, int nblocks)
{
    k_mass<T><<<nblocks, 256, 0, st>>>(D, wc, partial);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ batched step
//
// Many domains advance together: each stage is one launch over the blocks of
// all domains, and a per-stage block table gives every block its domain and
// its block coordinates inside that domain.  A block copies its domain's
// descriptor into shared memory and runs the same body as the single-domain
// kernel.  A domain whose controller has stopped it (t_end or step limit
// reached, or an error) has an inactive Coef: its blocks return at once.

// copy domain `dom`'s descriptor to shared memory (all threads of the block)
template <typename T>
__device__ __forceinline__ const Dev<T> &batch_dev(const Dev<T> *Ds, int dom)
{
    __shared__ __align__(16) unsigned long long sdev[(sizeof(Dev<T>) + 7) / 8];
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(Ds + dom);
    const int nthr = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int q = tid; q < (int)(sizeof(Dev<T>) / 8); q += nthr) sdev[q] = src[q];
    __syncthreads();
    return *reinterpret_cast<const Dev<T> *>(sdev);
}

// table entry: (domain, block of that domain, that domain's block count, 0)
template <typename T>
__global__ void __launch_bounds__(256) k_ghost_b(const Dev<T> *Ds, const int4 *tab)
{
    const int4 e = tab[blockIdx.x];
    const Dev<T> &D = batch_dev(Ds, e.x);
    ghost_body<T, MK_BATCH_MANY>(D, (long long)e.y * blockDim.x + threadIdx.x, (long long)e.z * blockDim.x);
}

// table entry: (domain, block of that domain, strips of 28 columns, 0)
template <typename T, int ROWS, bool THETA1, bool FAST, int YS = 0>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 2) k_rhs_sw_b(const Dev<T> *Ds, const int4 *tab)
{
    const int4 e = tab[blockIdx.x];
    const Dev<T> &D = batch_dev(Ds, e.x);
    rhs_sw_body<T, ROWS, THETA1, FAST, YS>(D, e.y, e.z);
}

// table entry: (domain, column group, chunk group, chunks per column)
template <typename T, int KY>
__global__ void __launch_bounds__(256) k_ysum_b(const Dev<T> *Ds, const int4 *tab)
{
    const int4 e = tab[blockIdx.x];
    const Dev<T> &D = batch_dev(Ds, e.x);
    ysum_body<T, KY>(D, e.y, e.z, e.w, D.ysums);
}

// table entry: (domain, block of that domain, chunks per column, 0)
template <typename T>
__global__ void __launch_bounds__(256) k_yscan_b(const Dev<T> *Ds, const int4 *tab)
{
    const int4 e = tab[blockIdx.x];
    const Dev<T> &D = batch_dev(Ds, e.x);
    yscan_body<T>(D, e.y, e.z, D.ysums, D.yin, D.yxa);
}

template <typename T, int KY>
__global__ void __launch_bounds__(256) k_yapply_b(const Dev<T> *Ds, const int4 *tab)
{
    const int4 e = tab[blockIdx.x];
    const Dev<T> &D = batch_dev(Ds, e.x);
    yapply_body<T, KY>(D, e.y, e.z, e.w, D.yin, D.yxa);
}

// table entry: (domain, block of that domain, that domain's block count,
// shared row length of the domain)
template <typename T, int K>
__global__ void __launch_bounds__(32 * XW_WARPS, sizeof(T) == 4 ? 4 : 2) k_xsolve_warp_b(const Dev<T> *Ds, const int4 *tab)
{
    const int4 e = tab[blockIdx.x];
    const Dev<T> &D = batch_dev(Ds, e.x);
    xsolve_warp_body<T, K>(D, e.y, (unsigned)e.z, e.w, 0.0);
}

// limits of the run and the controller of the first step, one thread per domain
template <typename T>
__global__ void k_batch_start(const Dev<T> *Ds, int n, const double *t_end, long long max_steps)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n) return;
    const Dev<T> &D = Ds[d];
    Ctl *ctl = D.ctl;
    ctl->t_end = t_end[d];
    ctl->n_limit = max_steps > 0 ? ctl->n + max_steps : 0x7fffffffffffffffLL;
    Coef cf;
    unsigned err;
    controller(D, 0.0, cf, err);
    *D.coef = cf;
    if (err) atomicOr(&ctl->err, err);
    ctl->done_count = 0u;
}

template <typename T>
__global__ void k_batch_gather(const Dev<T> *Ds, int n, Ctl *out)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < n) out[d] = *Ds[d].ctl;
}

// x-solver elements per thread of a batch (the default x_chunk, which also
// set every member's row pitch)
template <typename T>
int batch_xchunk()
{
    return sizeof(T) == 4 ? 8 : 4;
}

// table entry: (domain within the group, block of that domain, that domain's
// block count, its y row length); the group's descriptors are a kernel parameter
template <int K>
__global__ void __launch_bounds__(32 * XW_WARPS, 4) k_xsolve_warp_g(const __grid_constant__ RhsGroup G, const int4 *tab)
{
    const int4 e = tab[blockIdx.x];
    // the run-time switches stay here: compiled in, this kernel measured 3 % slower
    xsolve_warp_body<float, K>(G.d[e.x], e.y, (unsigned)e.z, e.w, 0.0);
}

template <typename T>
cudaError_t configure_batch(int yrow_max)
{
    const int bytes = XW_WARPS * yrow_max * (int)sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_xsolve_warp_b<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_xsolve_warp_b<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if constexpr (sizeof(T) == 4) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_xsolve_warp_g<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_xsolve_warp_g<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    }
    return e;
}

// table entry: (domain within the group, block of that domain, strips of 60
// columns, rows per warp); the group's descriptors are a kernel parameter
template <int YS>
__global__ void __launch_bounds__(128, 2) k_rhs_sw2_g(const __grid_constant__ RhsGroup G, const int4 *tab)
{
    const int4 e = tab[blockIdx.x];
    rhs_sw2_body<YS>(G.d[e.x], e.y, e.z, e.w);
}

template <typename T, int ROWS>
static void launch_batch_rhs(const Dev<T> *Ds, const BatchPlan &P, cudaStream_t st)
{
    if constexpr (sizeof(T) == 4) {
        if (P.rhs_pair) {
            for (int g = 0; g < P.rhs_ngroups; g++) {
                const int4 *tab = P.t_rhs + P.rhs_grp_off[g];
                if (P.ky == 16) k_rhs_sw2_g<16><<<P.rhs_grp_nb[g], 128, 0, st>>>(P.rhs_grp[g], tab);
                else k_rhs_sw2_g<8><<<P.rhs_grp_nb[g], 128, 0, st>>>(P.rhs_grp[g], tab);
            }
            return;
        }
    }
    if (P.rhs_fast && P.ky == 16) k_rhs_sw_b<T, ROWS, true, true, 16><<<P.nb_rhs, 128, 0, st>>>(Ds, P.t_rhs);
    else if (P.rhs_fast) k_rhs_sw_b<T, ROWS, true, true, 8><<<P.nb_rhs, 128, 0, st>>>(Ds, P.t_rhs);
    else if (P.rhs_theta1) k_rhs_sw_b<T, ROWS, true, false><<<P.nb_rhs, 128, 0, st>>>(Ds, P.t_rhs);
    else k_rhs_sw_b<T, ROWS, false, false><<<P.nb_rhs, 128, 0, st>>>(Ds, P.t_rhs);
}

template <typename T>
cudaError_t launch_batch_step(const Dev<T> *Ds, const BatchPlan &P, cudaStream_t st)
{
    k_ghost_b<T><<<P.nb_ghost, 256, sizeof(T) == 4 ? maker_step_bytes(P.ncomp_max) : 0, st>>>(Ds, P.t_ghost);
    if (P.rhs_rows == 32) launch_batch_rhs<T, 32>(Ds, P, st);
    else launch_batch_rhs<T, 64>(Ds, P, st);
    if (!P.rhs_fast) {  // (the fast RHS forms the chunk summaries itself)
        if (P.ky == 16) k_ysum_b<T, 16><<<P.nb_ysum, dim3(32, 8), 0, st>>>(Ds, P.t_ysum);
        else k_ysum_b<T, 8><<<P.nb_ysum, dim3(32, 8), 0, st>>>(Ds, P.t_ysum);
    }
    k_yscan_b<T><<<P.nb_yscan, 256, 0, st>>>(Ds, P.t_yscan);
    if (P.ky == 16) k_yapply_b<T, 16><<<P.nb_ysum, dim3(32, 8), 0, st>>>(Ds, P.t_ysum);
    else k_yapply_b<T, 8><<<P.nb_ysum, dim3(32, 8), 0, st>>>(Ds, P.t_ysum);
    const size_t xs = (size_t)XW_WARPS * P.yrow_max * sizeof(T);
    if constexpr (sizeof(T) == 4) {
        if (P.rhs_pair) {
            // descriptors as a kernel parameter, one launch per group (as the RHS stage)
            for (int g = 0; g < P.rhs_ngroups; g++) {
                const int4 *tab = P.t_x + P.x_grp_off[g];
                if (P.xk == 8) k_xsolve_warp_g<8><<<P.x_grp_nb[g], 32 * XW_WARPS, xs, st>>>(P.rhs_grp[g], tab);
                else k_xsolve_warp_g<4><<<P.x_grp_nb[g], 32 * XW_WARPS, xs, st>>>(P.rhs_grp[g], tab);
            }
            return cudaGetLastError();
        }
    }
    if (P.xk == 8) k_xsolve_warp_b<T, 8><<<P.nb_x, 32 * XW_WARPS, xs, st>>>(Ds, P.t_x);
    else k_xsolve_warp_b<T, 4><<<P.nb_x, 32 * XW_WARPS, xs, st>>>(Ds, P.t_x);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_start(const Dev<T> *Ds, int n, const double *t_end, long long max_steps, cudaStream_t st)
{
    k_batch_start<T><<<(n + 63) / 64, 64, 0, st>>>(Ds, n, t_end, max_steps);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_gather(const Dev<T> *Ds, int n, Ctl *out, cudaStream_t st)
{
    k_batch_gather<T><<<(n + 63) / 64, 64, 0, st>>>(Ds, n, out);
    return cudaGetLastError();
}

#define BSQ_INST(T)                                                                              \
    template int step_shape_ok<T>(int, int);                                                     \
    template int row_pitch<T>(int, int);                                                         \
    template int ysplit_chunks<T>(int, int);                                                     \
    template cudaError_t configure<T>(int);                                                      \
    template cudaError_t launch_step<T>(const Dev<T> &, cudaStream_t, double);                   \
    template cudaError_t launch_step_timed<T>(const Dev<T> &, cudaStream_t, double, cudaEvent_t *);\
    template cudaError_t launch_rate<T>(const Dev<T> &, cudaStream_t, int);                      \
    template cudaError_t launch_setup<T>(const Dev<T> &, cudaStream_t, const SetupArgs &);       \
    template cudaError_t launch_maker_table<T>(const Dev<T> &, cudaStream_t);                    \
    template cudaError_t launch_prologue<T>(const Dev<T> &, cudaStream_t, double, double, long long); \
    template int xsolver_staged<T>(const Dev<T> &, int);                                         \
    template int step_launches<T>(const Dev<T> &);                                               \
    template int batch_xchunk<T>();                                                              \
    template cudaError_t configure_batch<T>(int);                                                \
    template cudaError_t launch_batch_step<T>(const Dev<T> *, const BatchPlan &, cudaStream_t);  \
    template cudaError_t launch_batch_start<T>(const Dev<T> *, int, const double *, long long, cudaStream_t); \
    template cudaError_t launch_batch_gather<T>(const Dev<T> *, int, Ctl *, cudaStream_t);       \
    template cudaError_t launch_extract<T>(const Dev<T> &, cudaStream_t, int, int, T *);         \
    template cudaError_t launch_extract_f64<T>(const Dev<T> &, cudaStream_t, int, int, double *); \
    template cudaError_t launch_mass<T>(const Dev<T> &, cudaStream_t, int, double *, int);
BSQ_INST(float)
BSQ_INST(double)

}  // namespace bsq
