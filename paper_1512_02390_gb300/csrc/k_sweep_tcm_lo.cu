// Compile-time-window tcgen05 sweeps for the windows m = 5 ... 17 (levels p = 2, 4, 8);
// the kernel and its launch are in k_sweep_tc.cuh.
#include "k_sweep_tc.cuh"

namespace sem {

template <typename TIn>
cudaError_t sweep_tcm_lo(const DirView<float>& dx, const DirView<float>& dy, const TIn* r, float* E, int mode,
                         const float* nu_inv, const TcWork& wk, cudaStream_t s) {
  if constexpr (std::is_same<TIn, float>::value)
    return sweep_tcm_set<TIn, 5, 7, 9, 11, 13, 15, 17>(dx, dy, r, E, mode, nu_inv, wk, s);
  else
    return cudaErrorNotSupported;
}

template cudaError_t sweep_tcm_lo<float>(const DirView<float>&, const DirView<float>&, const float*, float*, int,
        const float*, const TcWork&, cudaStream_t);
template cudaError_t sweep_tcm_lo<double>(const DirView<float>&, const DirView<float>&, const double*, float*, int,
        const float*, const TcWork&, cudaStream_t);

}  // namespace sem
