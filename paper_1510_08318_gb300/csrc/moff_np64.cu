// Instantiation of the forward and adjoint MOFF kernels for N_p = 64.
#include "moff_fwd.cuh"
#include "moff_bwd.cuh"

namespace epic {

cudaError_t launch_fwd_64(int vdt, const SegList& L, int n_sm, cudaStream_t st, bool xpol) {
    switch (vdt) {
        case 0: return xpol ? launch_fwd_t<64, 0, true>(L, n_sm, st) : launch_fwd_t<64, 0>(L, n_sm, st);
        case 1: return xpol ? launch_fwd_t<64, 1, true>(L, n_sm, st) : launch_fwd_t<64, 1>(L, n_sm, st);
        case 2: return xpol ? launch_fwd_t<64, 2, true>(L, n_sm, st) : launch_fwd_t<64, 2>(L, n_sm, st);
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

int resident_fwd_workers_64(int vdt, int max_ant, int n_sm) {
    switch (vdt) {
        case 0: return resident_fwd_workers_t<64, 0>(max_ant, n_sm);
        case 1: return resident_fwd_workers_t<64, 1>(max_ant, n_sm);
        case 2: return resident_fwd_workers_t<64, 2>(max_ant, n_sm);
        default: return 0;
    }
}

}  // namespace epic
