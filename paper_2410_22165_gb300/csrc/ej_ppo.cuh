// PPO update: shared declarations.
#pragma once

#include "ej_policy.cuh"

namespace ej {

// Statistics accumulated per minibatch (doubles).
enum { ST_ADV_SUM = 0, ST_ADV_SQ = 1, ST_PG = 2, ST_VF = 3, ST_ENT = 4, ST_CLIP = 5, ST_KL = 6, ST_LOSS = 7, ST_COUNT_ = 8 };

// Minibatch m of an epoch: positions [lo, lo + count) of the Feistel
// permutation of [0, N) keyed by (k0, k1, ctr).
struct MbDesc {
    int lo, count;
    uint32_t N;
    int bits;          // the permutation's domain is [0, 2^bits), 2^bits >= N
    uint32_t k0, k1, ctr;
};

// Feistel permutation of [0, 2^bits) restricted to [0, N) by cycle walking
// (Luby-Rackoff; Black-Rogaway).  Alternating (unbalanced) form: the high
// part has bits / 2 bits, the low part the rest; each round replaces the
// part that is not the round function's input by its XOR with the round
// function (Philox word x0 of the other part, masked to the replaced
// part's width) and swaps the parts, so after the four rounds the widths
// are back in place.  With bits even this is the balanced network.
__device__ __forceinline__ uint32_t feistel(uint32_t x, int bits, uint32_t k0, uint32_t k1, uint32_t ctr) {
    const int wa = bits >> 1, wb = bits - wa;
    uint32_t A = x >> wb, B = x & ((1u << wb) - 1u);
    int la = wa, lb = wb;
#pragma unroll
    for (uint32_t rnd = 0; rnd < 4; ++rnd) {
        const uint32_t m = (1u << la) - 1u;
        const uint32_t F = philox4x32_10(make_uint4(B, rnd, ctr, 4u), k0, k1).x & m;
        const uint32_t nB = (A ^ F) & m;
        A = B;
        B = nB;
        const int t = la;
        la = lb;
        lb = t;
    }
    return (A << wb) | B;
}

__device__ __forceinline__ uint32_t mb_row(const MbDesc& d, int j) {
    uint32_t x = feistel((uint32_t)(d.lo + j), d.bits, d.k0, d.k1, d.ctr);
    while (x >= d.N) x = feistel(x, d.bits, d.k0, d.k1, d.ctr);
    return x;
}

// f(j, mb_row(d, j)) for j = j0, j0 + stride, ... < d.count, in that order.
// Each iteration applies the Feistel network once; a lane whose cycle walk
// has landed in [0, N) moves on to its next position, so the lanes of a warp
// stay busy while their walks differ in length.
template <class F>
__device__ __forceinline__ void mb_rows_strided(const MbDesc& d, int j0, int stride, F&& f) {
    int j = j0;
    uint32_t x = (uint32_t)(d.lo + j);
    while (j < d.count) {
        x = feistel(x, d.bits, d.k0, d.k1, d.ctr);
        if (x < d.N) {
            f(j, x);
            j += stride;
            x = (uint32_t)(d.lo + j);
        }
    }
}

struct FbArgs {
    MbDesc mb;
    int in_dim, in_pad, H, O, n_heads, head, W;
    float clip, vf_coef, vclip, ent_coef;
    const float* weights;
    const float* x;             // [N][in] rollout inputs (flat rows)
    const uint32_t* mask;       // [N][W] or NULL
    uint32_t* rows;             // [count] minibatch row table (BF16 path), or NULL
    const int32_t* act;         // [N][n_heads]
    const float* logp_old;      // [N]
    const float* v_old;         // [N]
    const float* adv;           // [N]
    const float* ret;           // [N]
    float* w3t; float* w2t; float* v2t;       // transposed weights (workspace)
    double* stats;              // [ST_COUNT_]
    const double* moments;      // NULL, or {count, sum, sum of squares} of the advantages over all ranks
    float* ws_x; float* ws_h1; float* ws_h2; float* ws_g1; float* ws_g2;
    float* ws_dl; float* ws_dz2; float* ws_dz1; float* ws_dy2; float* ws_dy1; float* ws_dv;
    // Per-agent population networks (Section 5; float32 path only): agents > 0
    // makes the minibatch the positions [lo, lo + count) of the permutation of
    // the T x E (step, environment) pairs, taken for every agent (rollout row
    // = position * agents + agent), tiles of one agent, per-agent advantage
    // moments (agent_moments[2 i], [2 i + 1]: sum, sum of squares), agent i's
    // actor at weights + i * actor_stride, critic at + i * critic_stride
    // (0: one shared critic, whose loss is the mean over all agents' rows),
    // transposed weights per agent (w3t + i * O * H, w2t + i * H * H,
    // v2t + i * H * H when the critic is per agent).  Per-row buffers hold
    // agent i's rows at [i * count, (i + 1) * count).
    int agents;
    size_t actor_stride, critic_stride;
    const double* agent_moments;
};

// Rows [0, nvalid) of a tile buffer to rows [base, base + nvalid) of a per-row buffer.
// dst[base + r][c] = buf[r][c] for the tile's first nvalid rows (dst row
// pitch ncols); 16-byte copies when ncols is a multiple of 4 and dst is
// 16-byte aligned (ld is a multiple of 4 at every call).
template <int ROWS = TILE>
__device__ inline void store_tile(const float* buf, int ld, int ncols, float* dst, int base, int nvalid) {
    if ((ncols & 3) == 0 && ((uintptr_t)dst & 15) == 0) {
        tile_for<ROWS>(ncols >> 2, [&](int r, int c4) {
            if (r < nvalid)
                *reinterpret_cast<float4*>(dst + (size_t)(base + r) * ncols + 4 * c4) =
                    *reinterpret_cast<const float4*>(buf + r * ld + 4 * c4);
        });
    } else {
        tile_for<ROWS>(ncols, [&](int r, int c) {
            if (r < nvalid) dst[(size_t)(base + r) * ncols + c] = buf[r * ld + c];
        });
    }
}

// out[r][c] = ref[r][c] > 0 ? out[r][c] : 0  (ReLU derivative); ncols and ld
// multiples of 4, out and ref 16-byte aligned.
template <int ROWS = TILE>
__device__ inline void mask_tile(float* out, int ld, const float* ref, int ncols) {
    tile_for<ROWS>(ncols >> 2, [&](int r, int c4) {
        float4* o = reinterpret_cast<float4*>(out + r * ld + 4 * c4);
        const float4 g = *reinterpret_cast<const float4*>(ref + r * ld + 4 * c4);
        float4 v = *o;
        if (!(g.x > 0.0f)) v.x = 0.0f;
        if (!(g.y > 0.0f)) v.y = 0.0f;
        if (!(g.z > 0.0f)) v.z = 0.0f;
        if (!(g.w > 0.0f)) v.w = 0.0f;
        *o = v;
    });
}

constexpr int WG_STRIDE = 128 * 128 + 128;   // floats of one job's partial up to hidden 128
// Floats of one job's partial sums (weights m x n, then the n bias sums) for
// the six gradient jobs of a network with `in` inputs, H hidden units and O
// logits: the largest m n + n of the jobs.
__host__ __device__ inline size_t wg_stride(int in, int H, int O) {
    size_t s = (size_t)in * H + H, t = (size_t)H * H + H, u = (size_t)H * O + O;
    s = s > t ? s : t;
    s = s > u ? s : u;
    return s > (size_t)WG_STRIDE ? s : (size_t)WG_STRIDE;
}
constexpr int WG_TILE = 128;                  // output rows / columns of one weight-gradient block
struct WgJob {
    const float* A; const float* B;
    int lda, ldb, m, n;
    long long w_off, b_off;      // where the weight and bias gradients go in the gradient vector
    // groups of rows with gradients of their own (per-agent networks): group g
    // is rows [g * group_rows, (g + 1) * group_rows) and adds to the gradient
    // at + g * w_gstride; groups = 0 means one group of all rows
    int groups, group_rows;
    long long w_gstride;
};
struct WgJobs { WgJob job[6]; };

size_t fwd_bwd_smem(int in_pad, int H, int O);
ej_status launch_gae(const float* rew, const float* value, const uint8_t* done, int T, int rows,
                     int per_env, float gamma, float lam, float* adv, float* ret, cudaStream_t s);
ej_status launch_minibatch_grad(const FbArgs& fa, const WgJobs& jobs, int n_jobs, float* partial,
                                size_t stride, int chunks, const float* w2, const float* w3, const float* v2,
                                float* grad, cudaStream_t s);
// Per-agent advantage moments of a grouped minibatch into moments[2 * agents].
ej_status launch_agent_moments(const MbDesc& mb, int agents, const float* adv, double* moments, cudaStream_t s);
// BF16 tensor-core minibatch gradient (ej_ppo_bf16.cu): advantage statistics,
// the fused kernel and the reduction into grad; partial: scratch of
// partial_bytes for the per-CTA accumulators.
ej_status launch_ppo_bf16(const FbArgs& fa, float* partial, size_t partial_bytes, float* grad, cudaStream_t s);
int ppo_bf16_fault(int clear);
// The minibatch loss of Section 4 from the gradient launch's sums, into
// stats[ST_LOSS]: (policy loss + vf_coef value loss - ent_coef entropy) / n,
// n = the minibatch's rows, or moments[0] (device) for the union of the
// ranks' minibatches of a data-parallel update.
ej_status launch_minibatch_loss(double* stats, int count, const double* moments, float vf_coef, float ent_coef,
                                cudaStream_t s);
// EJ_ERR_ARG unless every rollout-buffer array the call reads is present
// (net: EJ_NET_POP, EJ_NET_GOV or -1 for both; gae: GAE inputs; grad:
// minibatch-gradient inputs).
ej_status check_rollout(const EjRollout* b, int net, bool gae, bool grad);
// EJ_ERR_UNSUPPORTED when the float32 gradient's tile of network net (-1: both) exceeds shared memory.
// The BF16 gradient's shape limits (hidden, inputs, logits, heads, mask words).
ej_status bf16_grad_shape(int in_dim, int H, int O, int n_heads, int W);
ej_status check_grad_shape(const KParams& kp, int H, int precision, int net);
ej_status launch_adv_stats(const MbDesc& mb, const float* adv, double* stats, cudaStream_t s);
// Writes the minibatch's rollout rows (the permutation, once) and their advantage sums.
ej_status launch_mb_rows_stats(const MbDesc& mb, const float* adv, uint32_t* rows, double* stats, cudaStream_t s);
ej_status launch_adam(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                      float eps, int step, cudaStream_t s);

}  // namespace ej
