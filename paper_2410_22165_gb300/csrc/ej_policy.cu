// Policy forward and masked action sampling, float32 on the CUDA cores.
//
// Actor and critic are the 2 x H MLPs of Section 4 (ReLU hidden layers), one
// set of weights shared by all population agents and one for the government.
// A CTA takes tiles of 64 rows (agents; 32 where 64 do not fit shared
// memory); the activations of a tile stay in
// shared memory from the observation to the sampled action; weights are read
// through the L1 cache.  The sampler draws from the masked softmax (Section 3
// "Action masking": forbidden actions have probability zero) by inverse CDF.
#include <cfloat>
#include <cmath>

#include "ej_internal.cuh"
#include "ej_policy.cuh"

namespace ej {

namespace {

// Tiles of FTILE rows: 64 (thread tiles of 8 x 4, two CTAs per SM) wherever
// the tile fits shared memory, else 32 (4 x 4, at most 80 registers, up to
// three CTAs per SM).  The sampler takes one thread per row, so the larger
// tile samples twice the rows per pass (measured faster at 409,600 rows).
template <int FTILE, int MIN_BLOCKS>
__global__ void __launch_bounds__(NTH, MIN_BLOCKS) policy_fp32_kernel(PolicyArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int H = a.H, O = a.O, in_dim = a.in_dim;
    const int ldx = a.in_pad, ldh = H + 4, ldo = O + 1;
    float* xs = sm;                                  // [FTILE][ldx]
    float* hA = xs + FTILE * ldx;                     // [FTILE][ldh]
    float* hB = hA + FTILE * ldh;                     // [FTILE][ldh]
    float* lg = hB + FTILE * ldh;                     // [FTILE][ldo]
    float* val = lg + FTILE * ldo;                    // [FTILE]
    float* wsc = val + FTILE;                         // [FTILE][ldo] sampler scratch
    const NetOffsets off = net_offsets(in_dim, H, O);
    // shared networks: tiles of FTILE consecutive rows; per-agent networks:
    // tiles of one agent over FTILE consecutive environments
    const int n_env = a.rows / a.per_env;
    const int tpa = (n_env + FTILE - 1) / FTILE;
    const int n_tiles = a.agents ? a.agents * tpa : (a.rows + FTILE - 1) / FTILE;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int agent = a.agents ? tile / tpa : 0;
        const int e0 = a.agents ? (tile % tpa) * FTILE : 0;
        auto row_of = [&](int r) -> int {     // the tile's r-th row, or -1 past the end
            if (a.agents) return e0 + r < n_env ? (e0 + r) * a.per_env + agent : -1;
            const int row = tile * FTILE + r;
            return row < a.rows ? row : -1;
        };
        const float* wa = a.weights + (size_t)agent * a.actor_stride;
        const float* wc = a.weights + (size_t)agent * a.critic_stride;
        // observations of the tile (zero rows past the end, zero padding columns)
        tile_for<FTILE>(ldx, [&](int r, int k) {
            const int row = row_of(r);
            xs[r * ldx + k] = (row >= 0 && k < in_dim) ? a.x[(size_t)row * in_dim + k] : 0.0f;
        });
        __syncthreads();
        // actor: two hidden layers and the logits
        dense_tile<FTILE, FTILE / 8>(xs, ldx, in_dim, wa + off.W1, wa + off.b1, H, hA, ldh, true);
        __syncthreads();
        dense_tile<FTILE, FTILE / 8>(hA, ldh, H, wa + off.W2, wa + off.b2, H, hB, ldh, true);
        __syncthreads();
        head_tile<FTILE>(hB, ldh, H, wa + off.W3, wa + off.b3, O, lg, ldo);
        __syncthreads();
        // critic
        dense_tile<FTILE, FTILE / 8>(xs, ldx, in_dim, wc + off.V1, wc + off.c1, H, hA, ldh, true);
        __syncthreads();
        dense_tile<FTILE, FTILE / 8>(hA, ldh, H, wc + off.V2, wc + off.c2, H, hB, ldh, true);
        __syncthreads();
        value_tile<FTILE>(hB, ldh, H, wc + off.V3, wc[off.c3], val);
        __syncthreads();
        // sampling, one thread per row
        if (threadIdx.x < FTILE) {
            const int r = threadIdx.x, row = row_of(r);
            if (row >= 0) sample_row(a, row, lg + r * ldo, val[r], wsc + r * ldo);
        }
        __syncthreads();
    }
}

template <int FTILE>
size_t fp32_tile_smem(int in_pad, int H, int O) {
    return sizeof(float) * ((size_t)FTILE * in_pad + 2 * (size_t)FTILE * (H + 4) + 2 * (size_t)FTILE * (O + 1) + FTILE);
}

template <int FTILE, int MIN_BLOCKS>
ej_status launch_fp32_tiles(const PolicyArgs& a, size_t smem, cudaStream_t stream) {
    static SmemOptIn opt_in;     // per instantiation, per device
    ej_status st = opt_in.ensure((const void*)policy_fp32_kernel<FTILE, MIN_BLOCKS>, smem);
    if (st != EJ_OK) return st;
    const int n_tiles = a.agents ? a.agents * ((a.rows / a.per_env + FTILE - 1) / FTILE) : (a.rows + FTILE - 1) / FTILE;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, policy_fp32_kernel<FTILE, MIN_BLOCKS>, NTH, smem) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int cap = per_sm * device_sms();
    int grid = n_tiles < cap ? n_tiles : cap;
    if (grid < 1) grid = 1;
    policy_fp32_kernel<FTILE, MIN_BLOCKS><<<grid, NTH, smem, stream>>>(a);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "policy kernel launch: %s", cudaGetErrorString(err));
    return EJ_OK;
}

}  // namespace

size_t policy_fp32_smem(int in_pad, int H, int O) {
    const size_t s64 = fp32_tile_smem<64>(in_pad, H, O);
    return s64 <= 227u * 1024u ? s64 : fp32_tile_smem<32>(in_pad, H, O);
}

ej_status launch_policy_fp32(const PolicyArgs& a, cudaStream_t stream) {
    const size_t s64 = fp32_tile_smem<64>(a.in_pad, a.H, a.O);
    if (s64 <= 227u * 1024u) return launch_fp32_tiles<64, 2>(a, s64, stream);
    const size_t s32 = fp32_tile_smem<32>(a.in_pad, a.H, a.O);
    if (s32 > 227u * 1024u)
        return fail(EJ_ERR_UNSUPPORTED, "float32 policy: %d inputs, hidden %d and %d logits need %zu bytes of shared "
                    "memory per 32-row tile (at most %u)", a.in_pad, a.H, a.O, s32, 227u * 1024u);
    return launch_fp32_tiles<32, 3>(a, s32, stream);
}

}  // namespace ej
