// dp_fwd_minmax.cu -- forward sweep of the search for the paper's min-max (mjac) objective.
#include "dp_forward.cuh"

namespace cppflow {

cudaError_t launch_forward_minmax(const SingleSrc& s, int n, int nreq, int max_Kp, int form,
                              int cpc, cudaStream_t st) {
  return launch_forward_t<1>(s, n, nreq, max_Kp, form, cpc, st);
}
cudaError_t launch_forward_minmax(const BatchSrc& s, int n, int nreq, int max_Kp, int form,
                              int cpc, cudaStream_t st) {
  return launch_forward_t<1>(s, n, nreq, max_Kp, form, cpc, st);
}

}  // namespace cppflow
