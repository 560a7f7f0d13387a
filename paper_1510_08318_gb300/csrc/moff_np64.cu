// Instantiation of the forward and adjoint MOFF kernels for N_p = 64.
#include "moff_fwd.cuh"
#include "moff_bwd.cuh"

namespace epic {

cudaError_t launch_fwd_64(int vdt, const SegList& L, int n_sm, cudaStream_t st) {
    switch (vdt) {
        case 0: return launch_fwd_t<64, 0>(L, n_sm, st);
        case 1: return launch_fwd_t<64, 1>(L, n_sm, st);
        case 2: return launch_fwd_t<64, 2>(L, n_sm, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bwd_64(int vdt, const BwdArgs& a, int n_sm, cudaStream_t st) {
    switch (vdt) {
        case 0: return launch_bwd_t<64, 0>(a, n_sm, st);
        case 1: return launch_bwd_t<64, 1>(a, n_sm, st);
        case 2: return launch_bwd_t<64, 2>(a, n_sm, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace epic
