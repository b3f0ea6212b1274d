// Policy forward and masked action sampling, float32 on the CUDA cores.
//
// Actor and critic are the 2 x H MLPs of Section 4 (ReLU hidden layers), one
// set of weights shared by all population agents and one for the government.
// A CTA takes tiles of 64 rows (agents); the activations of a tile stay in
// shared memory from the observation to the sampled action; weights are read
// through the L1 cache.  The sampler draws from the masked softmax (Section 3
// "Action masking": forbidden actions have probability zero) by inverse CDF.
#include <cfloat>
#include <cmath>

#include "ej_internal.cuh"
#include "ej_policy.cuh"

namespace ej {

namespace {

__global__ void __launch_bounds__(NTH, 2) policy_fp32_kernel(PolicyArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int H = a.H, O = a.O, in_dim = a.in_dim;
    const int ldx = a.in_pad, ldh = H + 4, ldo = O + 1;
    float* xs = sm;                                  // [TILE][ldx]
    float* hA = xs + TILE * ldx;                     // [TILE][ldh]
    float* hB = hA + TILE * ldh;                     // [TILE][ldh]
    float* lg = hB + TILE * ldh;                     // [TILE][ldo]
    float* val = lg + TILE * ldo;                    // [TILE]
    float* wsc = val + TILE;                         // [TILE][ldo] sampler scratch
    const NetOffsets off = net_offsets(in_dim, H, O);
    // shared networks: tiles of TILE consecutive rows; per-agent networks:
    // tiles of one agent over TILE consecutive environments
    const int n_env = a.rows / a.per_env;
    const int tpa = (n_env + TILE - 1) / TILE;
    const int n_tiles = a.agents ? a.agents * tpa : (a.rows + TILE - 1) / TILE;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int agent = a.agents ? tile / tpa : 0;
        const int e0 = a.agents ? (tile % tpa) * TILE : 0;
        auto row_of = [&](int r) -> int {     // the tile's r-th row, or -1 past the end
            if (a.agents) return e0 + r < n_env ? (e0 + r) * a.per_env + agent : -1;
            const int row = tile * TILE + r;
            return row < a.rows ? row : -1;
        };
        const float* wa = a.weights + (size_t)agent * a.actor_stride;
        const float* wc = a.weights + (size_t)agent * a.critic_stride;
        // observations of the tile (zero rows past the end, zero padding columns)
        tile_for<TILE>(ldx, [&](int r, int k) {
            const int row = row_of(r);
            xs[r * ldx + k] = (row >= 0 && k < in_dim) ? a.x[(size_t)row * in_dim + k] : 0.0f;
        });
        __syncthreads();
        // actor: two hidden layers and the logits
        dense_tile(xs, ldx, in_dim, wa + off.W1, wa + off.b1, H, hA, ldh, true);
        __syncthreads();
        dense_tile(hA, ldh, H, wa + off.W2, wa + off.b2, H, hB, ldh, true);
        __syncthreads();
        head_tile(hB, ldh, H, wa + off.W3, wa + off.b3, O, lg, ldo);
        __syncthreads();
        // critic
        dense_tile(xs, ldx, in_dim, wc + off.V1, wc + off.c1, H, hA, ldh, true);
        __syncthreads();
        dense_tile(hA, ldh, H, wc + off.V2, wc + off.c2, H, hB, ldh, true);
        __syncthreads();
        value_tile(hB, ldh, H, wc + off.V3, wc[off.c3], val);
        __syncthreads();
        // sampling, one thread per row
        if (threadIdx.x < TILE) {
            const int r = threadIdx.x, row = row_of(r);
            if (row >= 0) sample_row(a, row, lg + r * ldo, val[r], wsc + r * ldo);
        }
        __syncthreads();
    }
}

}  // namespace

size_t policy_fp32_smem(int in_pad, int H, int O) {
    return sizeof(float) * ((size_t)TILE * in_pad + 2 * (size_t)TILE * (H + 4) + 2 * (size_t)TILE * (O + 1) + TILE);
}

ej_status launch_policy_fp32(const PolicyArgs& a, cudaStream_t stream) {
    const size_t smem = policy_fp32_smem(a.in_pad, a.H, a.O);
    if (smem > 227u * 1024u)
        return fail(EJ_ERR_UNSUPPORTED, "float32 policy: %d inputs, hidden %d and %d logits need %zu bytes of shared "
                    "memory per %d-row tile (at most %u)", a.in_pad, a.H, a.O, smem, TILE, 227u * 1024u);
    static SmemOptIn opt_in;
    ej_status st = opt_in.ensure((const void*)policy_fp32_kernel, smem);
    if (st != EJ_OK) return st;
    const int n_tiles = a.agents ? a.agents * ((a.rows / a.per_env + TILE - 1) / TILE) : (a.rows + TILE - 1) / TILE;
    const int cap = 2 * device_sms();
    int grid = n_tiles < cap ? n_tiles : cap;
    if (grid < 1) grid = 1;
    policy_fp32_kernel<<<grid, NTH, smem, stream>>>(a);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "policy kernel launch: %s", cudaGetErrorString(err));
    return EJ_OK;
}

}  // namespace ej
