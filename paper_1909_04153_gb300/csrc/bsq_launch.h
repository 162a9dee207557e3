// bsq_launch.h -- launchers of the step kernels (bsq_kernels.cu), called by
// the host engine (bsq_host.cu).  Internal to the library.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "bsq_internal.cuh"

namespace bsq {

template <typename T> int step_shape_ok(int nx, int ny);
template <typename T> int row_pitch(int nx, int tune);
template <typename T> int ysplit_chunks(int ny, int tune);
template <typename T> cudaError_t configure(int nx);
template <typename T> cudaError_t launch_step(const Dev<T> &D, cudaStream_t st, double forced_dt);
template <typename T> cudaError_t launch_step_timed(const Dev<T> &D, cudaStream_t st, double forced_dt, cudaEvent_t *ev);
template <typename T> int xsolver_staged(const Dev<T> &D, int nx);
template <typename T> int step_launches(const Dev<T> &D);
template <typename T>
cudaError_t launch_prologue(const Dev<T> &D, cudaStream_t st, double forced_dt, double t_end, long long max_steps);
template <typename T> cudaError_t launch_rate(const Dev<T> &D, cudaStream_t st, int wc);
template <typename T> cudaError_t launch_setup(const Dev<T> &D, cudaStream_t st, const SetupArgs &A);
template <typename T> cudaError_t launch_maker_table(const Dev<T> &D, cudaStream_t st);
template <typename T> cudaError_t launch_extract(const Dev<T> &D, cudaStream_t st, int wc, int field, T *out);
template <typename T> cudaError_t launch_extract_f64(const Dev<T> &D, cudaStream_t st, int wc, int field, double *out);
template <typename T> cudaError_t launch_mass(const Dev<T> &D, cudaStream_t st, int wc, double *partial, int nblocks);
cudaError_t launch_fma64(double *out, int blocks, int n, cudaStream_t st);  // 256 threads a block

// batched steps over many domains (one launch per stage)
template <typename T> int batch_xchunk();
template <typename T> cudaError_t configure_batch(int yrow_max);
template <typename T> cudaError_t launch_batch_step(const Dev<T> *Ds, const BatchPlan &P, cudaStream_t st);
template <typename T>
cudaError_t launch_batch_start(const Dev<T> *Ds, int n, const double *t_end, long long max_steps, cudaStream_t st);
template <typename T> cudaError_t launch_batch_gather(const Dev<T> *Ds, int n, Ctl *out, cudaStream_t st);

}  // namespace bsq
