// Compile-time-window tcgen05 sweeps for the windows m = 35, 37, 39 (p = 32),
// FP32 right sides; the kernel and its launch are in k_sweep_tc.cuh.
#include "k_sweep_tc.cuh"

namespace sem {

template <typename TIn>
cudaError_t sweep_tcm_p32(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E, int mode,
                          const float* nu_inv, const TcWork& wk, cudaStream_t s) {
  return sweep_tcm_set<TIn, 35, 37, 39>(dx, dy, r, E, mode, nu_inv, wk, s);
}

template cudaError_t sweep_tcm_p32<float>(const DirView<float>&, const DirView<float>&, const float*, float*, int,
        const float*, const TcWork&, cudaStream_t);

}  // namespace sem
