// bsq_host.cu -- host engine and C ABI (include/bsq.h) of the GB300 extended
// Boussinesq solver with variable-step AB3 time stepping (arXiv 1909.04153).
//
// bsq_create prepares everything that does not change in time: the bed at
// cell corners and centres (KP07 layout, Sec. 3), the still depth d and its
// gradients, the tridiagonal rows of Eqs. 19-21 with their boundary rows and
// their Thomas factors (the matrices depend on d only, so they are factored
// once), the sponge profiles and the wave-maker components.  bsq_advance then
// runs captured CUDA graphs of whole steps; the only host-device traffic per
// graph is the launch and a 64-byte status read.
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <new>
#include <thread>
#include <vector>

#include "../../include/bsq.h"
#include "bsq_internal.cuh"
#include "bsq_launch.h"

using namespace bsq;

struct bsq_domain {
    bsq_params p;
    bsq_boundary bnd;
    int fp64;
    int nx, ny, hx, pitch, rows;
    long long fstride;
    cudaStream_t stream;
    int own_stream;
    void *dmem;
    size_t dbytes;
    Ctl *ctl;
    Coef *coef;
    double *mass_partial;
    int mass_blocks;
    Ctl *h_ctl;  // pinned
    Dev<float> Df;
    Dev<double> Dd;
    cudaGraphExec_t graph;
    cudaGraphExec_t part[8];  // graphs of 1, 2, 4, ... steps below graph_steps (remainders)
    int graph_steps;
    int ctl_fresh;            // h_ctl equals the device Ctl (no work enqueued since it was read)
    bsq_status sticky;
    int n_state_fields;  // fields saved by a checkpoint
};

static const char *kStatus[] = {"ok", "invalid argument", "out of memory", "CUDA error",
                                "non-finite value in the state", "unstable: CFL step below dt_min",
                                "timed out waiting for the device", "invalid state"};

extern "C" const char *bsq_status_string(bsq_status s)
{
    if ((int)s < 0 || (int)s > 7) return "unknown status";
    return kStatus[(int)s];
}

extern "C" void bsq_params_default(bsq_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->g = 9.81;
    p->Bd = 1.0 / 15.0;
    p->cfl = 0.125;
    p->ema_alpha = 0.1;
    p->dt_min = 1e-9;
    p->theta = 1.0;
    p->timeout_s = 600.0;
    p->precision = BSQ_FP32;
    p->kahan = 1;
    p->cross_mode = BSQ_CROSS_SEQUENTIAL;
    p->graph_steps = 16;
}

#define CK(call)                                     \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) {                     \
            return BSQ_ERR_CUDA;                     \
        }                                            \
    } while (0)

static bsq_status set_sticky(bsq_domain *d, bsq_status s)
{
    if (d && d->sticky == BSQ_OK && s != BSQ_OK) d->sticky = s;
    return s;
}

// Bounded wait for a stream: polls cudaStreamQuery, yielding the thread
// between polls for the first 20 ms (a sleep overshoots by tens of
// microseconds, a few percent of a call of a few milliseconds) and sleeping
// 50 us between polls after that.
static bsq_status bounded_wait(cudaStream_t st, double lim)
{
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) return BSQ_OK;
        if (e != cudaErrorNotReady) return BSQ_ERR_CUDA;
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > lim) return BSQ_ERR_TIMEOUT;
        if (el < 20e-3) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Bounded wait for the domain's stream (limit_s <= 0: the domain's timeout).
static bsq_status wait_stream(const bsq_domain *d, double limit_s = 0.0)
{
    return bounded_wait(d->stream, limit_s > 0 ? limit_s : (d->p.timeout_s > 0 ? d->p.timeout_s : 600.0));
}

// Linearised dispersion relation of Eqs. 1-3 over still depth d:
// omega^2 = g d k^2 (1 + B (kd)^2) / (1 + (B + 1/3)(kd)^2); bisection on k
// (the right side increases with k).
static double wave_number(double omega, double d, double g, double B)
{
    if (omega <= 0.0 || d <= 0.0) return 0.0;
    auto f = [&](double k) {
        double kd2 = k * d * k * d;
        return g * d * k * k * (1.0 + B * kd2) / (1.0 + (B + 1.0 / 3.0) * kd2) - omega * omega;
    };
    double lo = 0.0, hi = omega / sqrt(g * d);
    while (f(hi) < 0.0) hi *= 2.0;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (f(mid) < 0.0) lo = mid; else hi = mid;
        if (hi - lo <= 1e-16 * hi) break;
    }
    return 0.5 * (lo + hi);
}

template <typename T>
static Dev<T> &dev_of(bsq_domain *d);
template <>
Dev<float> &dev_of<float>(bsq_domain *d) { return d->Df; }
template <>
Dev<double> &dev_of<double>(bsq_domain *d) { return d->Dd; }

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ------------------------------------------------------------------ create

// Byte offsets of everything in a domain's one device allocation.
struct Layout {
    size_t fb;  // bytes per padded field
    int nfields;
    size_t o_fields, o_corner, o_gx, o_gy, o_corr, o_cb, o_comp, o_mtab, o_ctl, o_coef, o_mass, o_ysum, total;
};
constexpr int kMassBlocks = 512;

template <typename T>
static Layout layout(int nx, int ny, int tune_xk, bool kahan, int nc)
{
    Layout L;
    const int pitch = row_pitch<T>(nx, tune_xk);
    const long long fs = (long long)pitch * (ny + 4);
    L.fb = align256((size_t)fs * sizeof(T));
    const int nstate = kahan ? 7 : 4;  // w0, w1, P, Q (+ cw, cP, cQ)
    L.nfields = nstate + 15 + 2 + 1 + 6 + (sizeof(T) == 8 ? 3 + ST_N : 0);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    L.o_fields = take(L.fb * L.nfields);
    L.o_corner = take((size_t)(nx + 5) * (ny + 5) * sizeof(T));
    L.o_gx = take((size_t)pitch * sizeof(T));  // row-length vector loads
    L.o_gy = take(ny * sizeof(T));
    L.o_corr = take((size_t)(4 * nx + 4 * ny + 4) * sizeof(T));
    L.o_cb = take((size_t)(2 * nx + 2 * ny) * sizeof(double));
    L.o_comp = take((size_t)7 * (nc > 0 ? nc : 1) * sizeof(double));
    // single precision: the maker's spatial-phase table, (cos, sin) per component
    // and maker point (the two ghost layers of all four sides, corners included)
    const size_t mpts = (size_t)4 * (ny + 4) + (size_t)4 * (nx + 4);
    L.o_mtab = take(sizeof(T) == 4 && nc > 0 ? mpts * nc * 2 * sizeof(float) : 0);
    L.o_ctl = take(sizeof(Ctl));
    L.o_coef = take(sizeof(Coef));
    L.o_mass = take(kMassBlocks * sizeof(double));
    // room for the smallest chunks, each column's count rounded up to 8
    const size_t nchy = (size_t)((ysplit_chunks<T>(ny, 8) + 7) & ~7) * nx;
    L.o_ysum = take(7 * nchy * sizeof(T));
    L.total = off;
    return L;
}

extern "C" size_t bsq_domain_bytes(const bsq_params *p, int n_comp)
{
    if (!p || p->nx < 3 || p->ny < 3 || p->nx > 16384 || p->ny > 16384) return 0;
    if (p->precision == BSQ_FP64) return layout<double>(p->nx, p->ny, p->tune[4], false, n_comp).total;
    return layout<float>(p->nx, p->ny, p->tune[4], p->kahan != 0, n_comp).total;
}


// The smallest double H with (H H)(H H) >= eps, each product rounded to
// double.  Rounding keeps order, so the rounded h^4 grows with h and, for
// h >= 0, h < H exactly when the rounded (h h)(h h) < eps: the near-dry test
// of the double-precision kernels compares h with H and forms h^4 only below
// it.  Bisection over the bit patterns of the non-negative doubles, which are
// ordered like the values.
static double dry_threshold(double eps)
{
    auto h4_reaches = [eps](uint64_t bits) {
        double h;
        memcpy(&h, &bits, sizeof h);
        volatile double h2 = h * h;
        volatile double h4 = h2 * h2;
        return h4 >= eps;
    };
    uint64_t lo = 0, hi = 0x7ff0000000000000ULL;  // +0 .. +inf, and inf^4 >= eps
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (h4_reaches(mid)) hi = mid;
        else lo = mid + 1;
    }
    double H;
    memcpy(&H, &lo, sizeof H);
    return H;
}

template <typename T>
static bsq_status create_T(bsq_domain *dm, const double *bed, const double *eta0, const double *P0,
                           const double *Q0)
{
    const bsq_params &p = dm->p;
    const int nx = p.nx, ny = p.ny;
    const int hx = 16 / (int)sizeof(T);
    const int pitch = row_pitch<T>(nx, p.tune[4]);  // covers hx + the x-solver's last chunk + 1
    const int rows = ny + 4;
    const long long fs = (long long)pitch * rows;
    // field stride: padded field rounded up to 256 bytes (the history ring is
    // indexed with this stride)
    const long long fstride = (long long)(align256((size_t)fs * sizeof(T)) / sizeof(T));
    dm->hx = hx;
    dm->pitch = pitch;
    dm->rows = rows;
    dm->fstride = fstride;
    if (!step_shape_ok<T>(nx, ny)) return BSQ_ERR_ARG;
    const bool kahan = p.kahan && sizeof(T) == 4;
    dm->p.kahan = kahan ? 1 : 0;

    // ---- static geometry, line factors and initial state are computed on the
    // device (launch_setup); the host keeps the per-side and per-line vectors
    const int cx = nx + 5;
    const int *bt = dm->bnd.type;
    for (int s = 0; s < 4; s++)
        if (bt[s] < BSQ_BC_WALL || bt[s] > BSQ_BC_MAKER) return BSQ_ERR_ARG;
    // still depth at cell (i, j), -1 <= i <= nx, -1 <= j <= ny, from the corner bed
    auto K = [&](int i, int j) {
        const int is = i < 0 ? -i : (i > nx ? 2 * nx - i : i);
        const int js = j < 0 ? -j : (j > ny ? 2 * ny - j : j);
        return bed[(size_t)is + (size_t)js * (nx + 1)];
    };
    auto D_ = [&](int i, int j) {
        const double bw = 0.5 * (K(i, j) + K(i, j + 1)), be = 0.5 * (K(i + 1, j) + K(i + 1, j + 1));
        const double bs = 0.5 * (K(i, j) + K(i + 1, j)), bn = 0.5 * (K(i, j + 1) + K(i + 1, j + 1));
        return fmax(p.w_s - 0.25 * (bw + be + bs + bn), 0.0);
    };
    // sponge profiles: gamma(r) = 1/2 + 1/2 cos(pi (1 - r/L)) inside a band of
    // width L, r from the outer edge; product over sponge sides
    auto sg = [](double r, double L) {
        if (L <= 0.0 || r >= L) return 1.0;
        if (r < 0.0) r = 0.0;
        return 0.5 + 0.5 * cos(M_PI * (1.0 - r / L));
    };
    std::vector<T> gx(nx), gy(ny);
    for (int i = 0; i < nx; i++) {
        double g = 1.0;
        if (bt[BSQ_WEST] == BSQ_BC_SPONGE) g *= sg((i + 0.5) * p.dx, dm->bnd.sponge_width[BSQ_WEST]);
        if (bt[BSQ_EAST] == BSQ_BC_SPONGE) g *= sg((nx - i - 0.5) * p.dx, dm->bnd.sponge_width[BSQ_EAST]);
        gx[i] = (T)g;
    }
    for (int j = 0; j < ny; j++) {
        double g = 1.0;
        if (bt[BSQ_SOUTH] == BSQ_BC_SPONGE) g *= sg((j + 0.5) * p.dy, dm->bnd.sponge_width[BSQ_SOUTH]);
        if (bt[BSQ_NORTH] == BSQ_BC_SPONGE) g *= sg((ny - j - 0.5) * p.dy, dm->bnd.sponge_width[BSQ_NORTH]);
        gy[j] = (T)g;
    }
    // wave-maker components at the still depth of the first maker side
    int nc = dm->bnd.n_comp;
    bool anymaker = false;
    for (int s = 0; s < 4; s++) anymaker |= bt[s] == BSQ_BC_MAKER;
    if (!anymaker) nc = 0;
    double dmk = 0.0;
    for (int s = 0; s < 4; s++) {
        if (bt[s] != BSQ_BC_MAKER) continue;
        int i = s == BSQ_WEST ? -1 : (s == BSQ_EAST ? nx : nx / 2);
        int j = s == BSQ_SOUTH ? -1 : (s == BSQ_NORTH ? ny : ny / 2);
        dmk = D_(i, j);
        break;
    }
    std::vector<double> comp((size_t)7 * (nc > 0 ? nc : 1), 0.0);
    for (int k = 0; k < nc; k++) {
        double om = 2.0 * M_PI * dm->bnd.freq[k];
        double kw = wave_number(om, dmk, p.g, p.Bd);
        double th = dm->bnd.dir[k];
        double c = kw > 0.0 ? om / kw : 0.0;
        comp[0 * nc + k] = dm->bnd.amp[k];
        comp[1 * nc + k] = om;
        comp[2 * nc + k] = kw * cos(th);
        comp[3 * nc + k] = kw * sin(th);
        comp[4 * nc + k] = dm->bnd.phase[k];
        comp[5 * nc + k] = c * cos(th);
        comp[6 * nc + k] = c * sin(th);
    }
    // ---- device memory: one allocation
    const Layout L = layout<T>(nx, ny, p.tune[4], kahan, nc);
    const size_t fb = L.fb;
    const size_t o_fields = L.o_fields, o_corner = L.o_corner, o_gx = L.o_gx, o_gy = L.o_gy, o_corr = L.o_corr;
    const size_t o_cb = L.o_cb, o_comp = L.o_comp, o_mtab = L.o_mtab, o_ctl = L.o_ctl, o_coef = L.o_coef;
    const size_t o_mass = L.o_mass;
    const size_t o_ysum = L.o_ysum, off = L.total;
    const int nstate = kahan ? 7 : 4;  // w0, w1, P, Q (+ cw, cP, cQ)
    const size_t nchy = (size_t)((ysplit_chunks<T>(ny, 8) + 7) & ~7) * nx;
    dm->mass_blocks = kMassBlocks;
    dm->dbytes = off;
    if (cudaMalloc(&dm->dmem, off) != cudaSuccess) { dm->dmem = nullptr; return BSQ_ERR_OOM; }
    char *base = (char *)dm->dmem;
    CK(cudaMemsetAsync(base, 0, off, dm->stream));
    Dev<T> &D = dev_of<T>(dm);
    memset(&D, 0, sizeof(D));
    D.nx = nx; D.ny = ny; D.pitch = pitch; D.hx = hx; D.fstride = fstride;
    D.dx = (T)p.dx; D.dy = (T)p.dy; D.rdx = (T)(1.0 / p.dx); D.rdy = (T)(1.0 / p.dy);
    D.dxd = p.dx; D.dyd = p.dy;
    D.g = (T)p.g; D.Bd = (T)p.Bd; D.w_s = (T)p.w_s; D.friction = (T)p.friction; D.theta = (T)p.theta;
    double eps = p.eps > 0.0 ? p.eps : pow(fmax(p.dx, p.dy), 4);
    D.eps = (T)eps;
    D.hdry = sizeof(T) == 8 ? (T)dry_threshold(eps) : (T)0;
    D.kahan = kahan ? 1 : 0;
    D.cross_mode = p.cross_mode;
    D.tune_rows = p.tune[3] == 16 || p.tune[3] == 24 || p.tune[3] == 32 || p.tune[3] == 48 || p.tune[3] == 64 ||
                          p.tune[3] == 128
                      ? p.tune[3]
                      : 0;
    D.tune_ysum = (p.tune[6] & 1) ? 1 : 0;
    D.tune_rhs1 = (p.tune[6] & 2) ? 1 : 0;
    D.tune_xtma = (p.tune[2] & 16) ? 4 : ((p.tune[2] & 8) ? 3 : ((p.tune[2] & 2) ? 1 : 0));
    D.tune_xk = (p.tune[4] == 4 || p.tune[4] == 8 || p.tune[4] == 16 || p.tune[4] == 32) ? p.tune[4] : 0;
    D.tune_yk = (p.tune[5] == 8 || p.tune[5] == 16) ? p.tune[5] : 0;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
            return BSQ_ERR_CUDA;
        D.nsm = nsm;
    }
    for (int s = 0; s < 4; s++) D.bc[s] = bt[s];
    D.cfl = p.cfl; D.ema_alpha = p.ema_alpha; D.dt_init = p.dt_init; D.dt_min = p.dt_min;
    D.dt_max = p.dt_max; D.ramp_time = p.ramp_time;
    T *F = (T *)(base + o_fields);
    auto field = [&](int k) { return (T *)((char *)F + fb * k); };
    int k = 0;
    D.w[0] = field(k++); D.w[1] = field(k++); D.P = field(k++); D.Q = field(k++);
    if (kahan) { D.cw = field(k++); D.cP = field(k++); D.cQ = field(k++); }
    else { D.cw = D.cP = D.cQ = nullptr; }
    D.hist = field(k); k += 15;
    D.dU = field(k++); D.dV = field(k++);
    D.bC = field(k++);
    D.fxm = field(k++); D.fxe = field(k++); D.fxc = field(k++);
    D.fym = field(k++); D.fye = field(k++); D.fyc = field(k++);
    if (sizeof(T) == 8) {
        D.fsc1 = field(k++); D.fsc2 = field(k++); D.fsc3 = field(k++);
        D.stat = field(k); k += ST_N;
        D.stat_stride = (long long)(fb / sizeof(T));
    } else {
        D.fsc1 = D.fsc2 = D.fsc3 = nullptr;
        D.stat = nullptr;
        D.stat_stride = 0;
    }
    D.corner = (T *)(base + o_corner);
    D.cpitch = cx;
    D.gx = (T *)(base + o_gx);
    D.gy = (T *)(base + o_gy);
    T *corr = (T *)(base + o_corr);
    D.corrW = corr; D.corrE = corr + ny; D.corrS = corr + 2 * ny; D.corrN = corr + 2 * ny + nx;
    T *mq = corr + 2 * ny + 2 * nx;
    D.mqW = mq; D.mqE = mq + ny; D.mqS = mq + 2 * ny; D.mqN = mq + 2 * ny + (nx + 2);
    double *cb = (double *)(base + o_cb);
    D.cW = cb; D.cE = cb + ny; D.cS = cb + 2 * ny; D.cN = cb + 2 * ny + nx;
    double *cp = (double *)(base + o_comp);
    D.ncomp = nc;
    D.amp = cp; D.om = cp + nc; D.kx = cp + 2 * nc; D.ky = cp + 3 * nc; D.ph = cp + 4 * nc;
    D.cx = cp + 5 * nc; D.cy = cp + 6 * nc;
    D.mtab = (sizeof(T) == 4 && nc > 0) ? (float2 *)(base + o_mtab) : nullptr;
    D.mpts = maker_points(D);
    D.ctl = (Ctl *)(base + o_ctl);
    D.coef = (Coef *)(base + o_coef);
    dm->ctl = D.ctl;
    dm->coef = D.coef;
    dm->mass_partial = (double *)(base + o_mass);
    // y-line chunk summaries (5 per chunk) and the scanned values entering and leaving each chunk
    D.ysums = (T *)(base + o_ysum);
    D.yin = D.ysums + 5 * nchy;
    D.yxa = D.ysums + 6 * nchy;
    dm->n_state_fields = nstate + 15;

    // device-side set-up from device copies of the caller's arrays: geometry,
    // Thomas factors (FP64, Eq. 21), initial state
    CK(cudaStreamSynchronize(dm->stream));
    {
        const size_t nbed = (size_t)(nx + 1) * (ny + 1), ncell = (size_t)nx * ny;
        const size_t nin = nbed + ncell * ((eta0 ? 1 : 0) + (P0 ? 1 : 0) + (Q0 ? 1 : 0));
        const size_t nscr = 2 * (size_t)fs;
        char *tmp = nullptr;
        const size_t tbytes = (nin + nscr) * sizeof(double) + 256;
        // stream-ordered scratch: no device-wide synchronisation (other domains may be running)
        if (cudaMallocAsync((void **)&tmp, tbytes, dm->stream) != cudaSuccess) return BSQ_ERR_OOM;
        double *dtmp = (double *)tmp;
        SetupArgs A;
        memset(&A, 0, sizeof(A));
        size_t o = 0;
        auto up = [&](const double *h, size_t n) -> const double * {
            if (!h) return nullptr;
            double *dst = dtmp + o;
            o += n;
            return cudaMemcpyAsync(dst, h, n * sizeof(double), cudaMemcpyHostToDevice, dm->stream) == cudaSuccess
                       ? dst
                       : nullptr;
        };
        A.bed = up(bed, nbed);
        A.eta0 = up(eta0, ncell);
        A.P0 = up(P0, ncell);
        A.Q0 = up(Q0, ncell);
        A.bCd = dtmp + o;
        A.dd = dtmp + o + fs;
        A.cW = cb; A.cE = cb + ny; A.cS = cb + 2 * ny; A.cN = cb + 2 * ny + nx;
        A.bad = (unsigned *)(tmp + (nin + nscr) * sizeof(double));
        A.w_s = p.w_s; A.Bd = p.Bd; A.dx = p.dx; A.dy = p.dy;
        for (int s = 0; s < 4; s++) A.bt[s] = bt[s] == BSQ_BC_MAKER ? MAKER : (bt[s] == BSQ_BC_SPONGE ? SPONGE : WALL);
        unsigned bad = 0;
        cudaError_t e = cudaMemsetAsync(A.bad, 0, sizeof(unsigned), dm->stream);
        if (e == cudaSuccess && (!A.bed || (eta0 && !A.eta0) || (P0 && !A.P0) || (Q0 && !A.Q0))) e = cudaErrorUnknown;
        if (e == cudaSuccess) e = launch_setup<T>(D, dm->stream, A);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, A.bad, sizeof(unsigned), cudaMemcpyDeviceToHost, dm->stream);
        cudaFreeAsync(tmp, dm->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(dm->stream);
        if (e != cudaSuccess) return BSQ_ERR_CUDA;
        if (bad) return BSQ_ERR_ARG;  // a line system is not diagonally dominant
    }
    CK(cudaMemcpy(D.gx, gx.data(), nx * sizeof(T), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(D.gy, gy.data(), ny * sizeof(T), cudaMemcpyHostToDevice));
    if (nc > 0) CK(cudaMemcpy(cp, comp.data(), comp.size() * sizeof(double), cudaMemcpyHostToDevice));
    CK(launch_maker_table<T>(D, dm->stream));
    Ctl c0;
    memset(&c0, 0, sizeof(c0));
    c0.t_end = INFINITY;
    c0.n_limit = 0x7fffffffffffffffLL;
    CK(cudaMemcpy(D.ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice));
    CK(configure<T>(nx));
    CK(launch_rate<T>(D, dm->stream, 0));
    return wait_stream(dm, 600.0);
}

extern "C" bsq_status bsq_create(const bsq_params *p, const double *bed_corners, const bsq_boundary *bnd,
                                 const double *eta0, const double *P0, const double *Q0, void *cuda_stream,
                                 bsq_domain **out)
{
    if (!out) return BSQ_ERR_ARG;
    *out = nullptr;
    if (!p || !bed_corners) return BSQ_ERR_ARG;
    if (p->nx < 3 || p->ny < 3 || p->nx > 16384 || p->ny > 16384) return BSQ_ERR_ARG;
    // cfl = 0: fixed steps of dt_init (the constant-step AB3 of Eqs. 16-18)
    if (!(p->cfl >= 0) || (p->cfl == 0 && !(p->dt_init > 0))) return BSQ_ERR_ARG;
    if (!(p->dx > 0) || !(p->dy > 0) || !(p->g > 0) || !(p->ema_alpha > 0) ||
        p->ema_alpha > 1.0 || p->Bd < 0 || (p->precision != BSQ_FP32 && p->precision != BSQ_FP64) ||
        (p->cross_mode != 0 && p->cross_mode != 1))
        return BSQ_ERR_ARG;
    bsq_boundary b;
    memset(&b, 0, sizeof(b));
    if (bnd) {
        b = *bnd;
        for (int s = 0; s < 4; s++)
            if (b.type[s] < 0 || b.type[s] > 2) return BSQ_ERR_ARG;
        bool maker = false;
        for (int s = 0; s < 4; s++) maker |= b.type[s] == BSQ_BC_MAKER;
        if (maker && (b.n_comp <= 0 || !b.amp || !b.freq || !b.phase || !b.dir)) return BSQ_ERR_ARG;
        if (b.n_comp < 0 || b.n_comp > BSQ_MAX_COMP) return BSQ_ERR_ARG;
    }
    cudaGetLastError();  // a failed call of another domain must not be reported here
    bsq_domain *d = new (std::nothrow) bsq_domain;
    if (!d) return BSQ_ERR_OOM;
    memset((void *)d, 0, sizeof(*d));
    d->p = *p;
    if (d->p.timeout_s <= 0) d->p.timeout_s = 600.0;
    d->graph_steps = p->graph_steps > 0 ? p->graph_steps : 16;
    d->bnd = b;
    // copy the component arrays (the caller's pointers are not kept)
    std::vector<double> comps;
    if (b.n_comp > 0 && b.amp) {
        comps.resize((size_t)4 * b.n_comp);
        memcpy(&comps[0], b.amp, b.n_comp * sizeof(double));
        memcpy(&comps[b.n_comp], b.freq, b.n_comp * sizeof(double));
        memcpy(&comps[2 * b.n_comp], b.phase, b.n_comp * sizeof(double));
        memcpy(&comps[3 * b.n_comp], b.dir, b.n_comp * sizeof(double));
        d->bnd.amp = &comps[0];
        d->bnd.freq = &comps[b.n_comp];
        d->bnd.phase = &comps[2 * b.n_comp];
        d->bnd.dir = &comps[3 * b.n_comp];
    }
    d->fp64 = p->precision == BSQ_FP64;
    d->nx = p->nx;
    d->ny = p->ny;
    if (cuda_stream) {
        d->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete d;
            return BSQ_ERR_CUDA;
        }
        d->own_stream = 1;
    }
    if (cudaMallocHost((void **)&d->h_ctl, sizeof(Ctl)) != cudaSuccess) {
        d->h_ctl = nullptr;
        bsq_destroy(d);
        return BSQ_ERR_OOM;
    }
    memset((void *)d->h_ctl, 0, sizeof(Ctl));  // t = 0, n = 0 until the first advance
    bsq_status st = d->fp64 ? create_T<double>(d, bed_corners, eta0, P0, Q0)
                            : create_T<float>(d, bed_corners, eta0, P0, Q0);
    d->bnd.amp = d->bnd.freq = d->bnd.phase = d->bnd.dir = nullptr;
    if (st != BSQ_OK) {
        bsq_destroy(d);
        return st;
    }
    *out = d;
    return BSQ_OK;
}

extern "C" void bsq_destroy(bsq_domain *d)
{
    if (!d) return;
    if (d->stream) cudaStreamSynchronize(d->stream);
    if (d->graph) cudaGraphExecDestroy(d->graph);
    for (int k = 0; k < 8; k++)
        if (d->part[k]) cudaGraphExecDestroy(d->part[k]);
    if (d->dmem) cudaFree(d->dmem);
    if (d->h_ctl) cudaFreeHost(d->h_ctl);
    if (d->own_stream && d->stream) cudaStreamDestroy(d->stream);
    delete d;
}

extern "C" size_t bsq_device_bytes(const bsq_domain *d) { return d ? d->dbytes : 0; }

// ------------------------------------------------------------------ stepping

// One step; its own dt was set by the previous step or the prologue, and
// forced_dt_next (> 0) fixes the next one.
static cudaError_t enqueue_step(bsq_domain *d, double forced_dt_next)
{
    return d->fp64 ? launch_step<double>(d->Dd, d->stream, forced_dt_next)
                   : launch_step<float>(d->Df, d->stream, forced_dt_next);
}

// Limits of the run, then the controller of the first step (forced_dt > 0:
// that step size).
static cudaError_t enqueue_start(bsq_domain *d, double t_end, long long max_steps, double forced_dt)
{
    return d->fp64 ? launch_prologue<double>(d->Dd, d->stream, forced_dt, t_end, max_steps)
                   : launch_prologue<float>(d->Df, d->stream, forced_dt, t_end, max_steps);
}

static bsq_status read_ctl(const bsq_domain *d)
{
    CK(cudaMemcpyAsync(d->h_ctl, d->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, d->stream));
    return wait_stream(d);
}

static bsq_status ctl_status(const Ctl &c)
{
    if (c.err & ERR_DEVICE_WAIT) return BSQ_ERR_TIMEOUT;
    if (c.err & ERR_NONFINITE) return BSQ_ERR_NONFINITE;
    if (c.err & (ERR_UNSTABLE | ERR_NODT)) return BSQ_ERR_UNSTABLE;
    return BSQ_OK;
}

// Capture `steps` steps into an executable graph.
static bsq_status capture_steps(bsq_domain *d, int steps, cudaGraphExec_t *out)
{
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < steps && e == cudaSuccess; s++) e = enqueue_step(d, 0.0);
    cudaError_t e2 = cudaStreamEndCapture(d->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) return BSQ_ERR_CUDA;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { *out = nullptr; return BSQ_ERR_CUDA; }
    return BSQ_OK;
}

// The graph of graph_steps steps and the remainder graphs of 1, 2, 4, ...
// steps below it (any remainder is at most a handful of graph launches).
static bsq_status build_graph(bsq_domain *d)
{
    if (d->graph) return BSQ_OK;
    bsq_status st = capture_steps(d, d->graph_steps, &d->graph);
    for (int k = 0; k < 8 && st == BSQ_OK && (1 << k) < d->graph_steps; k++)
        st = capture_steps(d, 1 << k, &d->part[k]);
    return st;
}

// Enqueue m step slots: whole graphs, then the remainder as its binary parts.
static bsq_status enqueue_slots(bsq_domain *d, long long m)
{
    for (long long r = 0; r < m / d->graph_steps; r++)
        if (cudaGraphLaunch(d->graph, d->stream) != cudaSuccess) return BSQ_ERR_CUDA;
    const long long rem = m % d->graph_steps;
    for (int k = 7; k >= 0; k--)
        if (rem & (1LL << k)) {
            cudaError_t e = d->part[k] ? cudaGraphLaunch(d->part[k], d->stream) : cudaErrorInvalidValue;
            if (e != cudaSuccess) return BSQ_ERR_CUDA;
        }
    return BSQ_OK;
}

// Steps a run to t_end probably still needs, from the last step size (the
// adaptive step changes slowly: Eq. 47 lets it rise gradually); -1 when there
// is no estimate (no finite end, or no step taken yet).
static long long steps_left_estimate(double t, double t_end, double last_dt)
{
    if (!isfinite(t_end) || !(last_dt > 0.0)) return -1;
    const double r = (t_end - t) / last_dt;
    if (!(r > 0.0)) return 1;
    return (long long)fmin(1.05 * r + 1.0, 1e15);
}

// How many step slots to enqueue before the next look at the controller
// state: the steps still allowed (budget), cut to the estimate of the steps
// left to t_end, without an estimate graph_steps x grow; at most 64 graphs.
static long long steps_to_enqueue(long long budget, long long est, int gs, int grow)
{
    long long want = budget;
    if (est > 0) want = est < want ? est : want;
    else if (budget == LLONG_MAX) want = (long long)gs * grow;
    const long long cap = 64LL * gs;
    return want < cap ? want : cap;
}

extern "C" bsq_status bsq_advance(bsq_domain *d, double t_end, long long max_steps, long long *steps_done)
{
    cudaGetLastError();  // a failed call of another domain must not be reported here
    if (steps_done) *steps_done = 0;
    if (!d) return BSQ_ERR_ARG;
    if (d->sticky != BSQ_OK) return d->sticky;
    if (isnan(t_end) || (max_steps <= 0 && !isfinite(t_end))) return BSQ_ERR_ARG;
    bsq_status st = BSQ_OK;
    if (!d->ctl_fresh) {  // (a call that ended with the controller state read needs no second read)
        st = read_ctl(d);
        if (st != BSQ_OK) return set_sticky(d, st);
    }
    const long long n0 = d->h_ctl->n;
    d->ctl_fresh = 0;
    if (cudaSuccess != enqueue_start(d, t_end, max_steps, 0.0)) return set_sticky(d, BSQ_ERR_CUDA);
    // Whole graphs of graph_steps steps, then the remainder in graphs of 1, 2,
    // 4, ... steps, so a call runs exactly the step slots it may need:
    // max_steps of them, or about the steps left to t_end (slots past the end
    // do no work).
    const double tol = isfinite(t_end) ? 1e-12 * fmax(1.0, fabs(t_end)) : 0.0;
    long long budget = max_steps > 0 ? max_steps : LLONG_MAX;
    int grow = 1;
    for (;;) {
        const long long est = steps_left_estimate(d->h_ctl->t, t_end, d->h_ctl->last_dt);
        const long long m = steps_to_enqueue(budget, est, d->graph_steps, grow);
        if (!d->graph) {
            // the domain's first run: these steps launch one by one, and the
            // graphs are captured and instantiated while the device runs them
            for (long long r = 0; r < m; r++)
                if (enqueue_step(d, 0.0) != cudaSuccess) return set_sticky(d, BSQ_ERR_CUDA);
            st = build_graph(d);
        } else {
            st = enqueue_slots(d, m);
        }
        if (st != BSQ_OK) return set_sticky(d, st);
        if (budget != LLONG_MAX) budget -= m;
        st = read_ctl(d);
        if (st != BSQ_OK) return set_sticky(d, st);
        st = ctl_status(*d->h_ctl);
        if (st != BSQ_OK) break;
        if (!(d->h_ctl->t < t_end - tol) || budget <= 0) break;
        if (grow < 64) grow *= 2;
    }
    if (steps_done) *steps_done = d->h_ctl->n - n0;
    d->ctl_fresh = 1;
    return set_sticky(d, st);
}

extern "C" bsq_status bsq_step_dt(bsq_domain *d, const double *dts, long long n)
{
    cudaGetLastError();  // a failed call of another domain must not be reported here
    if (!d || (n > 0 && !dts) || n < 0) return BSQ_ERR_ARG;
    if (d->sticky != BSQ_OK) return d->sticky;
    for (long long q = 0; q < n; q++)
        if (!(dts[q] > 0.0) || !isfinite(dts[q])) return BSQ_ERR_ARG;
    if (n == 0) return BSQ_OK;
    d->ctl_fresh = 0;
    if (cudaSuccess != enqueue_start(d, INFINITY, 0, dts[0])) return set_sticky(d, BSQ_ERR_CUDA);
    for (long long q = 0; q < n; q++) {
        if (enqueue_step(d, q + 1 < n ? dts[q + 1] : 0.0) != cudaSuccess) return set_sticky(d, BSQ_ERR_CUDA);
        if ((q & 255) == 255) {
            bsq_status st = read_ctl(d);
            if (st != BSQ_OK) return set_sticky(d, st);
            st = ctl_status(*d->h_ctl);
            if (st != BSQ_OK) return set_sticky(d, st);
        }
    }
    bsq_status st = read_ctl(d);
    if (st != BSQ_OK) return set_sticky(d, st);
    d->ctl_fresh = 1;
    return set_sticky(d, ctl_status(*d->h_ctl));
}

// ------------------------------------------------------------------ batches

struct bsq_batch {
    std::vector<bsq_domain *> doms;
    int fp64;
    cudaStream_t stream;
    int own_stream;
    void *dmem;          // descriptors, block tables, t_end, gathered Ctl
    void *Ds;            // Dev<T>[n]
    double *d_tend, *h_tend;
    Ctl *d_ctl, *h_ctl;  // gathered controller states (h_ctl pinned)
    BatchPlan plan;
    std::vector<RhsGroup> rhs_grp;          // descriptors of each RHS launch (single precision)
    std::vector<int> rhs_grp_nb, rhs_grp_off, x_grp_nb, x_grp_off;
    cudaGraphExec_t graph;
    int graph_stale;     // the block tables changed since the graph was captured
    int graph_steps;
    double timeout_s;
    size_t dcap;         // bytes of dmem
    int hcap;            // members the pinned host arrays hold
    int rows, xk, ky;    // tile shapes of the current tables
    int kahan, cross;    // the members' Kahan setting and cross mode
};

static bsq_status wait_batch(const bsq_batch *b) { return bounded_wait(b->stream, b->timeout_s); }

static void batch_free(bsq_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->dmem) cudaFree(b->dmem);
    if (b->h_tend) cudaFreeHost(b->h_tend);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

template <typename T> static constexpr bool pair_rhs() { return sizeof(T) == 4; }

// The block tables of every stage for the member domains with the given tile
// shapes (RHS rows per warp, x elements per lane, y rows per chunk); with the
// defaults each domain's blocks are laid out exactly as its own single-domain
// launches lay them out.
template <typename T>
static bsq_status batch_build(bsq_batch *b, int rows, int K, int KY)
{
    const int n = (int)b->doms.size();
    std::vector<int4> tg, tr, ts, tc, tx;
    bool fast = true, theta1 = true;
    // the tables are rewritten in place: no batched step may still read them
    // (the graph is captured again before the next launch)
    if (b->stream) CK(cudaStreamSynchronize(b->stream));
    b->graph_stale = 1;
    int yrow_max = 32 * K;
    std::vector<Dev<T>> hD(n);
    for (int d = 0; d < n; d++) {
        const Dev<T> &D = dev_of<T>(b->doms[d]);
        if (D.tune_yk != 0 || D.tune_xk != 0) return BSQ_ERR_ARG;
        fast = fast && D.theta == (T)1 && D.cross_mode != 0 && D.friction == (T)0 &&
               (D.kahan != 0) == (sizeof(T) == 4) && D.fstride * 15 < 0x7fffffffLL;
        theta1 = theta1 && D.theta == (T)1;
    }
    // the single-precision fast RHS pairs two columns per lane (strips of 60),
    // the others hold one column per lane (strips of 28)
    const bool pair = fast && pair_rhs<T>() && rows != 16;
    b->rhs_grp.clear();
    b->rhs_grp_nb.clear();
    b->rhs_grp_off.clear();
    b->x_grp_nb.clear();
    b->x_grp_off.clear();
    for (int d = 0; d < n; d++) {
        const Dev<T> &D = dev_of<T>(b->doms[d]);
        hD[d] = D;
        const int nx = D.nx, ny = D.ny;
        const long long nwork = 4LL * ny + 4LL * (nx + 4) + 2LL * ny + 2LL * nx;
        const int gb = (int)((nwork + 255) / 256);
        for (int q = 0; q < gb; q++) tg.push_back(make_int4(d, q, gb, 0));
        const int nstrip = pair ? (nx + 59) / 60 : (nx + 27) / 28, nband = (ny + rows - 1) / rows;
        const int rb = (int)(((long long)nstrip * nband + 3) / 4);
        // paired kernel: domains in groups of RHS_GROUP, one launch per group
        if (pair && d % RHS_GROUP == 0) {
            b->rhs_grp_off.push_back((int)tr.size());
            b->rhs_grp_nb.push_back(0);
        }
        for (int q = 0; q < rb; q++) tr.push_back(make_int4(pair ? d % RHS_GROUP : d, q, nstrip, rows));
        if (pair) b->rhs_grp_nb.back() += rb;
        const int nch = (ny + KY - 1) / KY;
        const int gx = (nx + 31) / 32, gy = (nch + 7) / 8;
        for (int by = 0; by < gy; by++)
            for (int bx = 0; bx < gx; bx++) ts.push_back(make_int4(d, bx, by, nch));
        const int cb = (int)(((long long)nx * 32 + 255) / 256);
        for (int q = 0; q < cb; q++) tc.push_back(make_int4(d, q, nch, 0));
        const int yrow = (nx + 32 * K - 1) / (32 * K) * (32 * K);
        if (yrow > yrow_max) yrow_max = yrow;
        const int xb = (ny + 3) / 4;
        if (pair && d % RHS_GROUP == 0) {
            b->x_grp_off.push_back((int)tx.size());
            b->x_grp_nb.push_back(0);
        }
        for (int q = 0; q < xb; q++) tx.push_back(make_int4(pair ? d % RHS_GROUP : d, q, xb, yrow));
        if (pair) b->x_grp_nb.back() += xb;
    }
    if ((size_t)4 * yrow_max * sizeof(T) > 96 * 1024) return BSQ_ERR_ARG;  // rows longer than the x-solver holds
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    const size_t o_D = take(n * sizeof(Dev<T>));
    const size_t o_g = take(tg.size() * sizeof(int4)), o_r = take(tr.size() * sizeof(int4));
    const size_t o_s = take(ts.size() * sizeof(int4)), o_c = take(tc.size() * sizeof(int4));
    const size_t o_x = take(tx.size() * sizeof(int4));
    const size_t o_t = take(n * sizeof(double)), o_ctl = take(n * sizeof(Ctl));
    if (off > b->dcap) {
        // grow (with room), keeping the old buffer until the new one exists
        void *nm = nullptr;
        const size_t cap = off + off / 2;
        if (cudaMalloc(&nm, cap) != cudaSuccess) return BSQ_ERR_OOM;
        if (b->dmem) cudaFree(b->dmem);
        b->dmem = nm;
        b->dcap = cap;
    }
    char *base = (char *)b->dmem;
    {
        // descriptors and all tables in one copy
        std::vector<char> h(o_t);
        memcpy(h.data() + o_D, hD.data(), n * sizeof(Dev<T>));
        memcpy(h.data() + o_g, tg.data(), tg.size() * sizeof(int4));
        memcpy(h.data() + o_r, tr.data(), tr.size() * sizeof(int4));
        memcpy(h.data() + o_s, ts.data(), ts.size() * sizeof(int4));
        memcpy(h.data() + o_c, tc.data(), tc.size() * sizeof(int4));
        memcpy(h.data() + o_x, tx.data(), tx.size() * sizeof(int4));
        CK(cudaMemcpyAsync(base, h.data(), o_t, cudaMemcpyHostToDevice, b->stream));
        CK(cudaStreamSynchronize(b->stream));
    }
    b->rows = rows;
    b->xk = K;
    b->ky = KY;
    b->Ds = base + o_D;
    b->d_tend = (double *)(base + o_t);
    b->d_ctl = (Ctl *)(base + o_ctl);
    BatchPlan &P = b->plan;
    P.n = n;
    P.nb_ghost = (int)tg.size(); P.nb_rhs = (int)tr.size(); P.nb_ysum = (int)ts.size();
    P.nb_yscan = (int)tc.size(); P.nb_x = (int)tx.size();
    P.t_ghost = (const int4 *)(base + o_g); P.t_rhs = (const int4 *)(base + o_r);
    P.t_ysum = (const int4 *)(base + o_s); P.t_yscan = (const int4 *)(base + o_c);
    P.t_x = (const int4 *)(base + o_x);
    P.rhs_fast = fast ? 1 : 0;
    P.rhs_pair = pair ? 1 : 0;
    P.rhs_ngroups = 0;
    if constexpr (sizeof(T) == 4) {
        if (pair) {
            const int ng = (n + RHS_GROUP - 1) / RHS_GROUP;
            b->rhs_grp.assign(ng, RhsGroup{});
            for (int d = 0; d < n; d++) b->rhs_grp[d / RHS_GROUP].d[d % RHS_GROUP] = hD[d];
            P.rhs_ngroups = ng;
        }
    }
    P.rhs_grp = b->rhs_grp.data();
    P.rhs_grp_nb = b->rhs_grp_nb.data();
    P.rhs_grp_off = b->rhs_grp_off.data();
    P.x_grp_nb = b->x_grp_nb.data();
    P.x_grp_off = b->x_grp_off.data();
    P.rhs_theta1 = theta1 ? 1 : 0;
    P.yrow_max = yrow_max;
    P.ncomp_max = 0;
    for (int d = 0; d < n; d++) P.ncomp_max = hD[d].ncomp > P.ncomp_max ? hD[d].ncomp : P.ncomp_max;
    P.rhs_rows = rows;
    P.xk = K;
    P.ky = KY;
    CK(configure_batch<T>(yrow_max));
    return BSQ_OK;
}

extern "C" bsq_status bsq_batch_create(bsq_domain *const *domains, int n, void *cuda_stream, bsq_batch **out)
{
    cudaGetLastError();
    if (!out) return BSQ_ERR_ARG;
    *out = nullptr;
    if (!domains || n < 1) return BSQ_ERR_ARG;
    for (int d = 0; d < n; d++) {
        bsq_domain *x = domains[d];
        if (!x || x->sticky != BSQ_OK) return BSQ_ERR_ARG;
        if (x->fp64 != domains[0]->fp64 || x->p.kahan != domains[0]->p.kahan ||
            x->p.cross_mode != domains[0]->p.cross_mode)
            return BSQ_ERR_ARG;
        for (int e = 0; e < d; e++)
            if (domains[e] == x) return BSQ_ERR_ARG;
    }
    bsq_batch *b = new (std::nothrow) bsq_batch();
    if (!b) return BSQ_ERR_OOM;
    b->doms.assign(domains, domains + n);
    b->fp64 = domains[0]->fp64;
    b->kahan = domains[0]->p.kahan;
    b->cross = domains[0]->p.cross_mode;
    b->graph_steps = domains[0]->graph_steps;
    b->timeout_s = 0.0;
    for (int d = 0; d < n; d++) {
        const double ts = domains[d]->p.timeout_s > 0 ? domains[d]->p.timeout_s : 600.0;
        if (ts > b->timeout_s) b->timeout_s = ts;
    }
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            b->stream = nullptr;
            batch_free(b);
            return BSQ_ERR_CUDA;
        }
        b->own_stream = 1;
    }
    if (cudaMallocHost((void **)&b->h_tend, n * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_ctl, n * sizeof(Ctl)) != cudaSuccess) {
        batch_free(b);
        return BSQ_ERR_OOM;
    }
    b->hcap = n;
    bsq_status st = b->fp64 ? batch_build<double>(b, 64, batch_xchunk<double>(), 8)
                            : batch_build<float>(b, 64, batch_xchunk<float>(), 8);
    if (st != BSQ_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return BSQ_OK;
}

extern "C" bsq_status bsq_batch_reset(bsq_batch *b, bsq_domain *const *domains, int n)
{
    cudaGetLastError();
    if (!b || !domains || n < 1) return BSQ_ERR_ARG;
    // (the previous members may have been destroyed already: only the batch's
    // own record of their settings is used)
    for (int d = 0; d < n; d++) {
        bsq_domain *x = domains[d];
        if (!x || x->sticky != BSQ_OK) return BSQ_ERR_ARG;
        if (x->fp64 != b->fp64 || x->p.kahan != b->kahan || x->p.cross_mode != b->cross) return BSQ_ERR_ARG;
        for (int e = 0; e < d; e++)
            if (domains[e] == x) return BSQ_ERR_ARG;
    }
    CK(cudaStreamSynchronize(b->stream));
    if (n > b->hcap) {
        double *ht = nullptr;
        Ctl *hc = nullptr;
        if (cudaMallocHost((void **)&ht, n * sizeof(double)) != cudaSuccess) return BSQ_ERR_OOM;
        if (cudaMallocHost((void **)&hc, n * sizeof(Ctl)) != cudaSuccess) {
            cudaFreeHost(ht);
            return BSQ_ERR_OOM;
        }
        cudaFreeHost(b->h_tend);
        cudaFreeHost(b->h_ctl);
        b->h_tend = ht;
        b->h_ctl = hc;
        b->hcap = n;
    }
    b->doms.assign(domains, domains + n);
    b->timeout_s = 0.0;
    for (int d = 0; d < n; d++) {
        const double ts = domains[d]->p.timeout_s > 0 ? domains[d]->p.timeout_s : 600.0;
        if (ts > b->timeout_s) b->timeout_s = ts;
    }
    return b->fp64 ? batch_build<double>(b, b->rows, b->xk, b->ky) : batch_build<float>(b, b->rows, b->xk, b->ky);
}

extern "C" void bsq_batch_destroy(bsq_batch *b) { batch_free(b); }

static bsq_status batch_read_ctl(bsq_batch *b)
{
    const int n = (int)b->doms.size();
    cudaError_t e = b->fp64 ? launch_batch_gather<double>((const Dev<double> *)b->Ds, n, b->d_ctl, b->stream)
                            : launch_batch_gather<float>((const Dev<float> *)b->Ds, n, b->d_ctl, b->stream);
    if (e != cudaSuccess) return BSQ_ERR_CUDA;
    CK(cudaMemcpyAsync(b->h_ctl, b->d_ctl, n * sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream));
    return wait_batch(b);
}

extern "C" bsq_status bsq_batch_advance(bsq_batch *b, const double *t_end, long long max_steps,
                                        long long *steps_done)
{
    cudaGetLastError();
    if (!b) return BSQ_ERR_ARG;
    const int n = (int)b->doms.size();
    if (steps_done)
        for (int d = 0; d < n; d++) steps_done[d] = 0;
    for (int d = 0; d < n; d++) {
        const double te = t_end ? t_end[d] : INFINITY;
        if (isnan(te) || (max_steps <= 0 && !isfinite(te))) return BSQ_ERR_ARG;
        b->h_tend[d] = te;
    }
    for (int d = 0; d < n; d++) {
        if (b->doms[d]->sticky != BSQ_OK) return b->doms[d]->sticky;
        b->doms[d]->ctl_fresh = 0;
        bsq_status s = wait_stream(b->doms[d]);  // the domain's own work comes first
        if (s != BSQ_OK) return set_sticky(b->doms[d], s);
    }
    bsq_status st = batch_read_ctl(b);
    if (st != BSQ_OK) return st;
    std::vector<long long> n0(n);
    for (int d = 0; d < n; d++) n0[d] = b->h_ctl[d].n;
    if (!b->graph || b->graph_stale) {
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int s = 0; s < b->graph_steps && e == cudaSuccess; s++)
            e = b->fp64 ? launch_batch_step<double>((const Dev<double> *)b->Ds, b->plan, b->stream)
                        : launch_batch_step<float>((const Dev<float> *)b->Ds, b->plan, b->stream);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) return BSQ_ERR_CUDA;
        // the same launch sequence with new grids and arguments: update the
        // executable graph in place; otherwise instantiate it again
        bool updated = false;
        if (b->graph) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(b->graph, g, &info) == cudaSuccess) {
                updated = true;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
            }
        }
        if (!updated) {
            e = cudaGraphInstantiate(&b->graph, g, 0);
            if (e != cudaSuccess) b->graph = nullptr;
        }
        cudaGraphDestroy(g);
        if (!b->graph) return BSQ_ERR_CUDA;
        b->graph_stale = 0;
    }
    CK(cudaMemcpyAsync(b->d_tend, b->h_tend, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    cudaError_t e = b->fp64
                        ? launch_batch_start<double>((const Dev<double> *)b->Ds, n, b->d_tend, max_steps, b->stream)
                        : launch_batch_start<float>((const Dev<float> *)b->Ds, n, b->d_tend, max_steps, b->stream);
    if (e != cudaSuccess) return BSQ_ERR_CUDA;
    // a domain is finished when it reached its t_end or its step limit, or failed
    auto all_done = [&]() {
        for (int d = 0; d < n; d++) {
            const Ctl &c = b->h_ctl[d];
            if (ctl_status(c) != BSQ_OK) continue;
            if (max_steps > 0 && c.n - n0[d] >= max_steps) continue;
            const double te = b->h_tend[d];
            const double tol = isfinite(te) ? 1e-12 * fmax(1.0, fabs(te)) : 0.0;
            if (c.t < te - tol) return false;
        }
        return true;
    };
    // whole graphs, then the remainder as single batched steps (as bsq_advance)
    long long budget = max_steps > 0 ? max_steps : LLONG_MAX;
    int grow = 1;
    for (;;) {
        long long est = -1;  // most steps any unfinished member probably still needs
        bool unknown = false;
        for (int d = 0; d < n; d++) {
            const Ctl &c = b->h_ctl[d];
            if (ctl_status(c) != BSQ_OK || (max_steps > 0 && c.n - n0[d] >= max_steps)) continue;
            const long long e = steps_left_estimate(c.t, b->h_tend[d], c.last_dt);
            if (e < 0) unknown = true;
            else if (e > est) est = e;
        }
        const long long m = steps_to_enqueue(budget, unknown ? -1 : est, b->graph_steps, grow);
        for (long long r = 0; r < m / b->graph_steps; r++)
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return BSQ_ERR_CUDA;
        for (long long r = 0; r < m % b->graph_steps; r++) {
            cudaError_t e2 = b->fp64 ? launch_batch_step<double>((const Dev<double> *)b->Ds, b->plan, b->stream)
                                     : launch_batch_step<float>((const Dev<float> *)b->Ds, b->plan, b->stream);
            if (e2 != cudaSuccess) return BSQ_ERR_CUDA;
        }
        if (budget != LLONG_MAX) budget -= m;
        st = batch_read_ctl(b);
        if (st != BSQ_OK) return st;
        if (all_done() || budget <= 0) break;
        if (grow < 64) grow *= 2;
    }
    bsq_status first = BSQ_OK;
    for (int d = 0; d < n; d++) {
        if (steps_done) steps_done[d] = b->h_ctl[d].n - n0[d];
        *b->doms[d]->h_ctl = b->h_ctl[d];
        b->doms[d]->ctl_fresh = 1;
        bsq_status s = ctl_status(b->h_ctl[d]);
        if (s != BSQ_OK) {
            set_sticky(b->doms[d], s);
            if (first == BSQ_OK) first = s;
        }
    }
    return first;
}

extern "C" int bsq_batch_size(const bsq_batch *b) { return b ? (int)b->doms.size() : 0; }

extern "C" int bsq_batch_launches_per_step(const bsq_batch *b)
{
    if (!b) return 0;
    // the fast RHS forms the y-line chunk summaries itself; with the paired RHS
    // the RHS and x-line stages are one launch per group of RHS_GROUP domains
    return (b->plan.rhs_fast ? 5 : 6) + (b->plan.rhs_pair ? 2 * (b->plan.rhs_ngroups - 1) : 0);
}

// Try every tile-shape combination on the batch itself (real steps), keep the
// fastest.
extern "C" bsq_status bsq_batch_autotune(bsq_batch *b, long long steps_per_trial, int *choice)
{
    if (!b || steps_per_trial < 1) return BSQ_ERR_ARG;
    const int n = (int)b->doms.size();
    const int ks_f[2] = {8, 4}, ks_d[1] = {4};
    const int *ks = b->fp64 ? ks_d : ks_f;
    const int nk = b->fp64 ? 1 : 2;
    const int rows_c[2] = {64, 32}, ky_c[2] = {8, 16};
    double best = 1e300;
    int br = 64, bk = ks[0], bky = 8;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<long long> done(n);
    bsq_status st = BSQ_OK;
    for (int ir = 0; ir < 2 && st == BSQ_OK; ir++)
        for (int ik = 0; ik < nk && st == BSQ_OK; ik++)
            for (int iy = 0; iy < 2 && st == BSQ_OK; iy++) {
                st = b->fp64 ? batch_build<double>(b, rows_c[ir], ks[ik], ky_c[iy])
                             : batch_build<float>(b, rows_c[ir], ks[ik], ky_c[iy]);
                if (st != BSQ_OK) break;
                st = bsq_batch_advance(b, nullptr, b->graph_steps, done.data());  // warm-up, builds the graph
                if (st != BSQ_OK) break;
                cudaEventRecord(e0, b->stream);
                st = bsq_batch_advance(b, nullptr, steps_per_trial, done.data());
                cudaEventRecord(e1, b->stream);
                if (st != BSQ_OK) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) { st = BSQ_ERR_CUDA; break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) { best = ms; br = rows_c[ir]; bk = ks[ik]; bky = ky_c[iy]; }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != BSQ_OK) return st;
    st = b->fp64 ? batch_build<double>(b, br, bk, bky) : batch_build<float>(b, br, bk, bky);
    if (st == BSQ_OK && choice) { choice[0] = br; choice[1] = bk; choice[2] = bky; }
    return st;
}

// ------------------------------------------------------------------ outputs

extern "C" bsq_status bsq_read_device(const bsq_domain *d, int field, void *dev_out)
{
    if (!d || !dev_out || field < 0 || field > 4) return BSQ_ERR_ARG;
    if (d->sticky != BSQ_OK && d->sticky != BSQ_ERR_NONFINITE && d->sticky != BSQ_ERR_UNSTABLE)
        return d->sticky;
    bsq_status st = read_ctl(d);
    if (st != BSQ_OK) return st;
    int wc = (int)(d->h_ctl->n & 1);
    cudaError_t e = d->fp64 ? launch_extract<double>(d->Dd, d->stream, wc, field, (double *)dev_out)
                            : launch_extract<float>(d->Df, d->stream, wc, field, (float *)dev_out);
    return e == cudaSuccess ? BSQ_OK : BSQ_ERR_CUDA;
}

extern "C" bsq_status bsq_read(const bsq_domain *d, int field, double *host_out)
{
    if (!d || !host_out || field < 0 || field > 4) return BSQ_ERR_ARG;
    if (d->sticky != BSQ_OK && d->sticky != BSQ_ERR_NONFINITE && d->sticky != BSQ_ERR_UNSTABLE)
        return d->sticky;
    const size_t ncell = (size_t)d->nx * d->ny;
    bsq_status st = read_ctl(d);
    if (st != BSQ_OK) return st;
    const int wc = (int)(d->h_ctl->n & 1);
    // widened to double on the device, then one copy into the caller's array
    double *tmp = nullptr;
    if (cudaMallocAsync((void **)&tmp, ncell * sizeof(double), d->stream) != cudaSuccess) return BSQ_ERR_OOM;
    cudaError_t e = d->fp64 ? launch_extract_f64<double>(d->Dd, d->stream, wc, field, tmp)
                            : launch_extract_f64<float>(d->Df, d->stream, wc, field, tmp);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, tmp, ncell * sizeof(double), cudaMemcpyDeviceToHost, d->stream);
    cudaFreeAsync(tmp, d->stream);
    bsq_status w = wait_stream(d);
    if (e != cudaSuccess) return BSQ_ERR_CUDA;
    return w;
}

extern "C" bsq_status bsq_info(const bsq_domain *d, double *t, long long *n, double *last_dt, double *mass,
                               long long *clamps)
{
    if (!d) return BSQ_ERR_ARG;
    bsq_status st = read_ctl(d);
    if (st != BSQ_OK) return st;
    Ctl c = *d->h_ctl;
    if (t) *t = c.t;
    if (n) *n = c.n;
    if (last_dt) *last_dt = c.last_dt;
    if (clamps) *clamps = (long long)c.clamps;
    if (mass) {
        int wc = (int)(c.n & 1);
        cudaError_t e = d->fp64 ? launch_mass<double>(d->Dd, d->stream, wc, d->mass_partial, d->mass_blocks)
                                : launch_mass<float>(d->Df, d->stream, wc, d->mass_partial, d->mass_blocks);
        if (e != cudaSuccess) return BSQ_ERR_CUDA;
        std::vector<double> part(d->mass_blocks);
        CK(cudaMemcpyAsync(part.data(), d->mass_partial, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                           d->stream));
        st = wait_stream(d);
        if (st != BSQ_OK) return st;
        double s = 0.0;
        for (double v : part) s += v;
        *mass = s * d->p.dx * d->p.dy;
    }
    return ctl_status(c) == BSQ_OK ? d->sticky : ctl_status(c);
}

extern "C" bsq_status bsq_clock(const bsq_domain *d, double *t, long long *n)
{
    if (!d) return BSQ_ERR_ARG;
    const Ctl &c = *d->h_ctl;
    if (t) *t = c.t;
    if (n) *n = c.n;
    if (d->sticky != BSQ_OK) return d->sticky;
    return ctl_status(c);
}

// ------------------------------------------------------------------ checkpoint

struct CkptHeader {
    char magic[8];
    int version, nx, ny, precision, kahan, cross_mode, nfields, pad;
    long long fstride;
};

static void state_ptrs(const bsq_domain *d, std::vector<void *> &ptrs, size_t &fbytes)
{
    if (d->fp64) {
        const Dev<double> &D = d->Dd;
        ptrs = {D.w[0], D.w[1], D.P, D.Q};
        for (int k = 0; k < 15; k++) ptrs.push_back(D.hist + (size_t)k * D.fstride);
        fbytes = (size_t)D.fstride * 8;
    } else {
        const Dev<float> &D = d->Df;
        ptrs = {D.w[0], D.w[1], D.P, D.Q};
        if (D.kahan) { ptrs.push_back(D.cw); ptrs.push_back(D.cP); ptrs.push_back(D.cQ); }
        for (int k = 0; k < 15; k++) ptrs.push_back(D.hist + (size_t)k * D.fstride);
        fbytes = (size_t)D.fstride * 4;
    }
}

extern "C" bsq_status bsq_checkpoint(const bsq_domain *d, void *buf, size_t *len)
{
    if (!d || !len) return BSQ_ERR_ARG;
    std::vector<void *> ptrs;
    size_t fbytes;
    state_ptrs(d, ptrs, fbytes);
    size_t need = sizeof(CkptHeader) + sizeof(Ctl) + ptrs.size() * fbytes;
    if (!buf) { *len = need; return BSQ_OK; }
    if (*len < need) { *len = need; return BSQ_ERR_ARG; }
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "BSQCKPT", 8);
    h.version = 1; h.nx = d->nx; h.ny = d->ny; h.precision = d->fp64; h.kahan = d->p.kahan;
    h.cross_mode = d->p.cross_mode; h.nfields = (int)ptrs.size(); h.fstride = d->fstride;
    char *o = (char *)buf;
    memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    CK(cudaMemcpyAsync(o, d->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, d->stream));
    o += sizeof(Ctl);
    for (void *p : ptrs) {
        CK(cudaMemcpyAsync(o, p, fbytes, cudaMemcpyDeviceToHost, d->stream));
        o += fbytes;
    }
    *len = need;
    return wait_stream(d);
}

extern "C" bsq_status bsq_restore(bsq_domain *d, const void *buf, size_t len)
{
    if (!d || !buf) return BSQ_ERR_ARG;
    std::vector<void *> ptrs;
    size_t fbytes;
    state_ptrs(d, ptrs, fbytes);
    size_t need = sizeof(CkptHeader) + sizeof(Ctl) + ptrs.size() * fbytes;
    if (len < need) return BSQ_ERR_ARG;
    CkptHeader h;
    memcpy(&h, buf, sizeof(h));
    if (memcmp(h.magic, "BSQCKPT", 8) != 0 || h.version != 1 || h.nx != d->nx || h.ny != d->ny ||
        h.precision != d->fp64 || h.kahan != d->p.kahan || h.nfields != (int)ptrs.size() ||
        h.fstride != d->fstride)
        return BSQ_ERR_ARG;
    const char *o = (const char *)buf + sizeof(h);
    bsq_status st = wait_stream(d);
    if (st != BSQ_OK) return st;
    d->ctl_fresh = 0;
    CK(cudaMemcpy(d->ctl, o, sizeof(Ctl), cudaMemcpyHostToDevice));
    o += sizeof(Ctl);
    for (void *p : ptrs) {
        CK(cudaMemcpy(p, o, fbytes, cudaMemcpyHostToDevice));
        o += fbytes;
    }
    d->sticky = BSQ_OK;
    return BSQ_OK;
}

// ------------------------------------------------------------------ profiling

static const char *kKernelNames[] = {"ghost", "rhs_combine", "ysolve", "xrhs", "xsolve"};

extern "C" const char *bsq_kernel_name(int k)
{
    return (k >= 0 && k < 5) ? kKernelNames[k] : "";
}

extern "C" bsq_status bsq_fp64_fma_rate(double *tflops)
{
    if (!tflops) return BSQ_ERR_ARG;
    *tflops = 0.0;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
        return BSQ_ERR_CUDA;
    const int blocks = 8 * nsm, n = 2048;  // 8 blocks of 256 threads a multiprocessor
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double *out = nullptr;
    bsq_status rc = BSQ_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
        cudaMalloc((void **)&out, (size_t)blocks * 256 * sizeof(double)) == cudaSuccess &&
        launch_fma64(out, blocks, n, st) == cudaSuccess &&  // warm-up
        cudaEventRecord(e0, st) == cudaSuccess && launch_fma64(out, blocks, n, st) == cudaSuccess &&
        cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
            *tflops = 2.0 * 8.0 * n * (double)blocks * 256.0 / (ms * 1e-3) / 1e12;
            rc = BSQ_OK;
        }
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return rc;
}

extern "C" bsq_status bsq_profile_kernels(bsq_domain *d, long long n_steps, double *ms_out, int *n_kernels)
{
    if (!d || !ms_out || !n_kernels || n_steps <= 0) return BSQ_ERR_ARG;
    if (d->sticky != BSQ_OK) return d->sticky;
    cudaEvent_t ev[6];
    for (int k = 0; k < 6; k++)
        if (cudaEventCreate(&ev[k]) != cudaSuccess) return BSQ_ERR_CUDA;
    for (int k = 0; k < 5; k++) ms_out[k] = 0.0;
    bsq_status st = BSQ_OK;
    d->ctl_fresh = 0;
    if (cudaSuccess != enqueue_start(d, INFINITY, n_steps, 0.0)) st = BSQ_ERR_CUDA;
    for (long long q = 0; q < n_steps && st == BSQ_OK; q++) {
        cudaError_t e = d->fp64 ? launch_step_timed<double>(d->Dd, d->stream, 0.0, ev)
                                : launch_step_timed<float>(d->Df, d->stream, 0.0, ev);
        if (e != cudaSuccess) { st = BSQ_ERR_CUDA; break; }
        st = wait_stream(d);
        if (st != BSQ_OK) break;
        for (int k = 0; k < 5; k++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) != cudaSuccess) { st = BSQ_ERR_CUDA; break; }
            ms_out[k] += ms;
        }
    }
    for (int k = 0; k < 6; k++) cudaEventDestroy(ev[k]);
    for (int k = 0; k < 5; k++) ms_out[k] /= (double)n_steps;
    *n_kernels = 5;
    if (st == BSQ_OK) {
        st = read_ctl(d);
        if (st == BSQ_OK) st = ctl_status(*d->h_ctl);
    }
    return set_sticky(d, st);
}

extern "C" int bsq_launches_per_step(const bsq_domain *d)
{
    if (!d) return 0;
    return d->fp64 ? step_launches<double>(d->Dd) : step_launches<float>(d->Df);
}
