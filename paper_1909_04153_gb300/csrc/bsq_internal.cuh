// bsq_internal.cuh -- device-side data structures and helpers of the GB300
// extended Boussinesq solver (arXiv 1909.04153).  Shared by the kernels and
// the host engine of the library; nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bsq {

enum { WALL = 0, SPONGE = 1, MAKER = 2 };
enum { SW = 0, SE = 1, SS = 2, SN = 3 };

// error flags raised on the device
enum : unsigned { ERR_NONFINITE = 1u, ERR_UNSTABLE = 2u, ERR_NODT = 4u, ERR_DEVICE_WAIT = 8u };

// Controller state of one domain (FP64, device resident).  The controller
// kernel reads it; the first block of the stencil kernel commits the step.
struct Ctl {
    double t;                 // simulated time of level n
    double dtm1, dtm2;        // dt_{n-1}, dt_{n-2}
    double t_end;             // advance target
    double last_dt;
    long long n;              // steps taken
    long long n_limit;        // no step starts once n >= n_limit
    unsigned long long rate_bits;  // Eq. 22 rate of the current state (bits of a positive double)
    unsigned long long clamps;     // positivity clamps so far
    unsigned int err;
    unsigned int done_count;  // x-solver blocks finished in the current step
};

// Per-step coefficients written by the controller, read by the step kernels.
struct Coef {
    int active;               // 1: this step does work
    int s0, s1, s2;           // ring slots of levels n, n-1, n-2
    int nlev;                 // history levels used (1: first Euler step, 2, 3)
    int wc;                   // index of the w buffer holding level n
    long long n;
    double t0, t1, dt;
    double ramp0, ramp1;      // wave-maker ramp r(t) at t_n and t_{n+1}
    double beta[3], gam[3];
    float betaf[3], gamf[3];
};

// Static terms of the double-precision RHS (Eqs. 11-13), formed at set-up from
// the corner bed and the still depth exactly as the kernel formed them:
// bed-slope source -g (b_E - b_W) / dx and the face-bed mean (b_E + b_W) / 2 in
// x, the same in y, and for the dispersive terms B g d^2, B g d^3 and the
// central differences d_x, d_y of the still depth.
enum { ST_SX = 0, ST_MX, ST_SY, ST_MY, ST_BD2, ST_BD3, ST_DDX, ST_DDY, ST_N };

// Everything a kernel needs, passed by value.  T = float or double.
template <typename T>
struct Dev {
    int nx, ny;
    int pitch;                // elements per padded row
    int hx;                   // halo columns left of the interior
    long long fstride;        // elements per padded field
    T dx, dy, rdx, rdy;       // cell sizes and reciprocals
    double dxd, dyd;          // cell sizes in FP64 (wave-maker phases)
    T g, Bd, eps, w_s, friction, theta;
    T hdry;                   // FP64: h < hdry exactly when (h h)(h h) < eps (the near-dry test of KP07)
    int kahan, cross_mode;
    int tune_rows;                 // RHS rows per warp (0: by grid size)
    int tune_xtma;                 // x-solver: 0 automatic, 1 registers only, 3 persistent, 4 warp per row
    int nsm;                       // multiprocessors of the device
    int tune_xk, tune_yk;          // x-solver elements per thread, split y-solver rows per chunk (0: default)
    int tune_ysum;                 // 1: chunk summaries by their own kernel, not in the RHS kernel
    int tune_rhs1;                 // 1: one column per lane in the sliding-window RHS (single precision)
    T *ysums, *yin, *yxa;          // its chunk summaries (5 per chunk) and scanned values
    int bc[4];
    // controller inputs (FP64)
    double cfl, ema_alpha, dt_init, dt_min, dt_max;
    double ramp_time;
    // state (padded fields with a 2-cell halo)
    T *w[2];                  // ping-pong water level
    T *cw, *P, *cP, *Q, *cQ;  // fluxes and compensation terms
    T *hist;                  // 5 fields x 3 levels, field f slot s at hist + (3 f + s) fstride
    T *dU, *dV;               // increments for the line solves (scratch)
    // static fields
    T *corner;                // bed at corners, (nx+5) x (ny+5), origin (-2,-2)
    int cpitch;
    T *bC;                    // bed at cell centres (padded field, halo included)
    T *fxm, *fxe, *fxc;       // x-line Thomas factors: m, -a m, c m
    T *fym, *fye, *fyc;       // y-line Thomas factors
    // double precision: the F*, G* coefficients of Eqs. 14-15 at the cell
    // centres, d d_x / 6, d d_y / 6 and (B + 1/3) d^2 (null in single precision)
    T *fsc1, *fsc2, *fsc3;
    // double precision: further static terms of the RHS at the cell centres,
    // field k at stat + k stat_stride (ST_*; null in single precision)
    T *stat;
    long long stat_stride;
    T *gx, *gy;               // sponge factor profiles along x and y (product of sides)
    const double *cW, *cE, *cS, *cN;  // raw boundary coefficients for maker rows
    T *corrW, *corrE, *corrS, *corrN; // per-step maker corrections of the line right-hand sides
    T *mqW, *mqE, *mqS, *mqN;         // maker Q at t_{n+1}: W/E per row, S/N per column -1..nx
    // wave maker
    int ncomp;
    const double *amp, *om, *kx, *ky, *ph, *cx, *cy;
    float2 *mtab;             // single precision: cos and sin of each component's spatial phase at
    int mpts;                 // the mpts maker points, [component][point] (null without a maker)
    // controller
    Ctl *ctl;
    Coef *coef;
};

// Inputs of the device-side set-up of a new domain (geometry, line factors,
// initial state): device copies of the caller's arrays and FP64 scratch.
struct SetupArgs {
    const double *bed;               // (nx+1) x (ny+1) corner elevations, row-major
    const double *eta0, *P0, *Q0;    // nx x ny, or null
    double *bCd, *dd;                // scratch: bed at centres and still depth, padded fields
    double *cW, *cE, *cS, *cN;       // boundary coefficients of the line systems (outputs)
    unsigned *bad;                   // set when a line is not diagonally dominant
    double w_s, Bd, dx, dy;
    int bt[4];                       // boundary type per side (W, E, S, N)
};

// Descriptors of up to RHS_GROUP member domains passed by value to one
// launch of the batched single-precision RHS kernel: kernel parameters live
// in the constant bank, which the kernel reads like the single-domain kernel
// reads its own descriptor (a copy in shared memory costs it registers).
constexpr int RHS_GROUP = 48;
struct RhsGroup {
    Dev<float> d[RHS_GROUP];
};

// Block tables of a batched step: entry b of a stage's table says which
// domain block b of that stage's single launch works on, and where (the
// meaning of the remaining fields is the stage's, see the batched kernels).
struct BatchPlan {
    int n;                                        // domains
    int nb_ghost, nb_rhs, nb_ysum, nb_yscan, nb_x;  // blocks of each stage's launch
    const int4 *t_ghost, *t_rhs, *t_ysum, *t_yscan, *t_x;
    int rhs_fast, rhs_theta1;                     // RHS variant shared by all domains
    int rhs_pair;                                 // single precision: two columns per lane (k_rhs_sw2 body)
    int rhs_ngroups;                              // with rhs_pair: launches of the RHS and x-line
    const RhsGroup *rhs_grp;                      // stages, and per launch (host arrays) its
    const int *rhs_grp_nb, *rhs_grp_off;          // descriptors, blocks and first entry in t_rhs
    const int *x_grp_nb, *x_grp_off;              // and in t_x
    int yrow_max;                                 // x-solver shared row length (elements)
    int ncomp_max;                                // most wave-maker components of a domain
    int rhs_rows, xk, ky;                         // tile shapes: RHS rows per warp, x elements per
                                                  // lane, y rows per chunk (the autotuner's knobs)
};

// Maker points of the single-precision maker table: two ghost layers on each
// of the four sides, each layer two cells longer than the side at either end.
template <typename T>
__host__ __device__ inline int maker_points(const Dev<T> &D)
{
    return 4 * (D.ny + 4) + 4 * (D.nx + 4);
}

template <typename T>
__host__ __device__ inline long long fidx(const Dev<T> &D, int i, int j)
{
    return (long long)(j + 2) * D.pitch + (i + D.hx);
}

__device__ inline unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ inline double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

}  // namespace bsq
