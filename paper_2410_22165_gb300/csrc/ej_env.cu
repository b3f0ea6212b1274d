// Generic instantiations of the environment kernel (resource and price-level
// counts read from the parameters) and the draw generator; the launcher
// dispatches the default market to its compile-time instantiation.
#include "ej_env.cuh"

namespace ej {

namespace {

__global__ void fill_draws_kernel(KParams p, uint32_t k0, uint32_t k1, uint32_t g0, int n_steps,
                                  int32_t* act, float* gather_u, uint32_t* tb, float* policy_u,
                                  int32_t* gov_act) {
    const size_t n_pop = (size_t)n_steps * p.E * p.A;
    const size_t n_gov = (size_t)n_steps * p.E;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_pop + n_gov; k += stride) {
        if (k < n_pop) {
            const uint32_t i = (uint32_t)(k % p.A);
            const size_t se = k / p.A;
            const uint32_t e = (uint32_t)(se % p.E);
            const uint32_t s = (uint32_t)(se / p.E);
            const uint4 x = philox4x32_10(make_uint4(i, e, g0 + s, 0u), k0, k1);
            if (act) act[k] = below(x.x, p.nA);
            if (gather_u) gather_u[k] = u01(x.y);
            if (tb) tb[k] = x.z;
            if (policy_u) policy_u[k] = u01(x.w);
        } else if (gov_act) {
            const size_t kg = k - n_pop;
            const uint32_t e = (uint32_t)(kg % p.E);
            const uint32_t s = (uint32_t)(kg / p.E);
            const uint4 x = philox4x32_10(make_uint4(0u, e, g0 + s, 1u), k0, k1);
            const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
            for (int b = 0; b < p.nb; ++b) gov_act[kg * p.nb + b] = below(xs[b], p.tax_levels);
        }
    }
}

}  // namespace

ej_status launch_env(const KParams& kp, const Layout& lay, const DevState& st, const DevIO& io,
                     int n_steps, int mode, uint64_t seed, cudaStream_t stream) {
    using envk::launch_nt;
    if (kp.R == 2 && lay.sizes.threads <= 512) {
        if (kp.P == 5) return launch_env_r2p5(kp, lay, st, io, n_steps, mode, seed, stream);
        if (kp.P == 10) return launch_env_r2p10(kp, lay, st, io, n_steps, mode, seed, stream);
        if (kp.P == 20) return launch_env_r2p20(kp, lay, st, io, n_steps, mode, seed, stream);
    }
    switch (lay.sizes.threads) {
        case 32: return launch_nt<32, 0, 0>(kp, lay, st, io, n_steps, mode, seed, stream);
        case 64: return launch_nt<64, 0, 0>(kp, lay, st, io, n_steps, mode, seed, stream);
        case 128: return launch_nt<128, 0, 0>(kp, lay, st, io, n_steps, mode, seed, stream);
        case 256: return launch_nt<256, 0, 0>(kp, lay, st, io, n_steps, mode, seed, stream);
        case 512: return launch_nt<512, 0, 0>(kp, lay, st, io, n_steps, mode, seed, stream);
        case 1024: return launch_nt<1024, 0, 0>(kp, lay, st, io, n_steps, mode, seed, stream);
        default: return fail(EJ_ERR_UNSUPPORTED, "no kernel for %d threads", lay.sizes.threads);
    }
}

ej_status launch_fill_draws(const KParams& kp, uint64_t seed, uint32_t g0, int n_steps,
                            int32_t* act, float* gather_u, uint32_t* tb, float* policy_u,
                            int32_t* gov_act, cudaStream_t stream) {
    const size_t total = (size_t)n_steps * kp.E * (kp.A + 1);
    int blocks = (int)((total + 255) / 256);
    if (blocks > device_sms() * 16) blocks = device_sms() * 16;
    if (blocks < 1) blocks = 1;
    fill_draws_kernel<<<blocks, 256, 0, stream>>>(kp, (uint32_t)seed, (uint32_t)(seed >> 32), g0, n_steps,
                                                  act, gather_u, tb, policy_u, gov_act);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "fill_draws launch: %s", cudaGetErrorString(err));
    return EJ_OK;
}

}  // namespace ej
