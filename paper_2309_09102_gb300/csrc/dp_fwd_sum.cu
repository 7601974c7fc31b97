// dp_fwd_sum.cu -- forward sweep of the search for summed per-step L-inf jumps.
#include "dp_forward.cuh"

namespace cppflow {

cudaError_t launch_forward_sum(const SingleSrc& s, int n, int nreq, int max_Kp, int form,
                              int cpc, cudaStream_t st) {
  return launch_forward_t<0>(s, n, nreq, max_Kp, form, cpc, st);
}
cudaError_t launch_forward_sum(const BatchSrc& s, int n, int nreq, int max_Kp, int form,
                              int cpc, cudaStream_t st) {
  return launch_forward_t<0>(s, n, nreq, max_Kp, form, cpc, st);
}

}  // namespace cppflow
