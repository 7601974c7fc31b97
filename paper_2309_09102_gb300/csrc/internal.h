// internal.h -- declarations shared by the library's translation units.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <math_constants.h>

#include "common.cuh"

namespace cppflow {

// fk_mask.cu
cudaError_t launch_mask(const SingleSrc& s, const cpp_params_t& P, cudaStream_t st);
cudaError_t launch_mask_batch(const BatchSrc& s, int n, int nreq, long long max_tasks,
                              const cpp_params_t& P, cudaStream_t st);
long long mask_tasks(int T, int Kp);
cudaError_t launch_fk_batch(const cpp_robot_t& r, const float* q, long long N, float* R,
                            float* p, cudaStream_t st);
cudaError_t launch_fk_pose64(const cpp_robot_t& r, const double* q, long long N, double* pose,
                             cudaStream_t st);

// dp.cu
int bp_stride(int Kp);
size_t dp_smem_bytes(int n, int Kp);
bool dp_supported(int n, int Kp);
cudaError_t launch_dp(const SingleSrc& s, unsigned stages, cudaStream_t st);
cudaError_t launch_dp_batch(const BatchSrc& s, unsigned stages, int n, int nreq, int max_T,
                            int max_Kp, cudaStream_t st);

// lm.cu
cudaError_t launch_lm(const SingleSrc& s, const cpp_params_t& P, bool want_err, cudaStream_t st);
cudaError_t launch_lm_batch(const BatchSrc& s, int nreq, int max_T, const cpp_params_t& P,
                            cudaStream_t st);
cudaError_t launch_check(const SingleSrc& s, const cpp_params_t& P, cudaStream_t st);
cudaError_t launch_check_batch(const BatchSrc& s, int nreq, const cpp_params_t& P,
                               cudaStream_t st);

}  // namespace cppflow
