// Environment kernel instantiations for markets of 2 resources and 10 price
// levels (44 population actions, 40 book levels), both counts known at
// compile time.
#include "ej_env.cuh"

namespace ej {

ej_status launch_env_r2p10(const KParams& kp, const Layout& lay, const DevState& st, const DevIO& io,
                          int n_steps, int mode, uint64_t seed, cudaStream_t stream) {
    using envk::launch_nt;
    if (kp.R != 2 || kp.P != 10) return fail(EJ_ERR_UNSUPPORTED, "2-resource, 10-level kernel called for R=%d P=%d", kp.R, kp.P);
    switch (lay.sizes.threads) {
        case 32: return launch_nt<32, 2, 10>(kp, lay, st, io, n_steps, mode, seed, stream);
        case 64: return launch_nt<64, 2, 10>(kp, lay, st, io, n_steps, mode, seed, stream);
        case 128: return launch_nt<128, 2, 10>(kp, lay, st, io, n_steps, mode, seed, stream);
        case 256: return launch_nt<256, 2, 10>(kp, lay, st, io, n_steps, mode, seed, stream);
        case 512: return launch_nt<512, 2, 10>(kp, lay, st, io, n_steps, mode, seed, stream);
        default: return fail(EJ_ERR_UNSUPPORTED, "no 2-resource, 10-level kernel for %d threads", lay.sizes.threads);
    }
}

}  // namespace ej
