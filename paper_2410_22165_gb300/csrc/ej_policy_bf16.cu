// Policy forward on the 5th-generation tensor cores: BF16 operands, FP32
// accumulation in tensor memory (tcgen05.mma, kind::f16, M = 128).
//
// One CTA per SM, persistent over tiles of 128 rows (thread i of the 4 warps
// owns row i, i.e. TMEM lane i).  At start the CTA packs the actor and
// critic weights into shared memory as K-major BF16 operands in the 128-byte
// swizzled layout.  Per tile: observations -> BF16 operand; layer 1 of actor
// and critic as one N = 2H MMA chain; epilogue (bias, ReLU, BF16) back into
// shared memory as the next operand; layer 2 of actor and critic; the two
// heads; the last epilogue adds the biases and samples the action with the
// same sampler as the float32 path.  Thread 0 issues the MMAs; completion is
// signalled through tcgen05.commit to an mbarrier; every wait is bounded.
#include <cfloat>
#include <cmath>

#include "ej_internal.cuh"
#include "ej_policy.cuh"
#include "ej_ppo.cuh"

namespace ej {
__device__ int g_ej_fault = 0;   // fault word of the bounded waits in this library
}

#include "ej_tc.cuh"

namespace ej {

namespace {

constexpr int BM = 128;     // rows per tile = TMEM lanes
constexpr int BT = 256;     // threads per CTA: two warpgroups share the 128 TMEM lanes
constexpr int KX = 64;      // observation width padded to one 64-element panel
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t COL_D3 = 256, COL_D4 = 384;

struct BfLayout {
    uint32_t w1, w2a, w2c, w3, v3, x, h, bias, vals, total;
    int N3;
};

__host__ __device__ inline BfLayout bf_layout(int H, int O) {
    BfLayout L;
    L.N3 = (O + 15) / 16 * 16;
    uint32_t b = 0;
    L.w1 = b;  b += 2u * H * KX * 2;           // [2H][KX]
    L.w2a = b; b += (uint32_t)H * H * 2;       // [H][H]
    L.w2c = b; b += (uint32_t)H * H * 2;
    L.w3 = b;  b += (uint32_t)L.N3 * H * 2;    // [N3][H]
    L.v3 = b;  b += 16u * H * 2;               // [16][H]
    L.x = b;   b += BM * KX * 2;               // [BM][KX]
    L.h = b;   b += BM * 2u * H * 2;           // [BM][2H]; later logits + sampler scratch
    L.bias = b; b += ((4u * H + (uint32_t)O + 4) * 4 + 1023) & ~1023u;   // b1|c1, b2|c2, b3, c3
    L.vals = b; b += BM * 4;
    L.total = b;
    return L;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void st_shared_v4(uint8_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(p)), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Packs rows x K of a K-major operand from a float source: element (n, k) =
// get(n, k).  Work items (chunk of 8 k, row n), rows fastest.
template <class F>
__device__ void pack_operand(uint8_t* dst, int rows, int K, F get) {
    // Items (8 consecutive k of row n) four at a time: all their loads are
    // issued before any conversion and store, so a thread waits for memory
    // once per four items rather than once per item.
    constexpr int G = 4;
    const int items = rows * (K / 8);
    const int step = (int)blockDim.x;
    for (int it0 = threadIdx.x; it0 < items; it0 += G * step) {
        float v[G][8];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int it = it0 + g * step;
            const int n = it % rows, kc = it / rows;
#pragma unroll
            for (int q = 0; q < 8; ++q) v[g][q] = it < items ? get(n, kc * 8 + q) : 0.0f;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int it = it0 + g * step;
            if (it < items) {
                const int n = it % rows, kc = it / rows;
                st_shared_v4(dst + sw128_offset(n, kc * 8, rows), pack2(v[g][0], v[g][1]), pack2(v[g][2], v[g][3]),
                             pack2(v[g][4], v[g][5]), pack2(v[g][6], v[g][7]));
            }
        }
    }
}

// 32 accumulator columns of this thread's row -> bias, ReLU, BF16 -> operand
// columns [k0, k0 + 32) of row `row` in the swizzled [BM][K] operand.
__device__ __forceinline__ void epilogue32(uint32_t taddr, const float* bias, uint8_t* dst, int row, int k0) {
    float v[32];
    tmem_ld32(taddr, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 b0 = *reinterpret_cast<const float4*>(bias + q * 8);
        const float4 b1 = *reinterpret_cast<const float4*>(bias + q * 8 + 4);
        const float y0 = fmaxf(v[q * 8 + 0] + b0.x, 0.0f), y1 = fmaxf(v[q * 8 + 1] + b0.y, 0.0f);
        const float y2 = fmaxf(v[q * 8 + 2] + b0.z, 0.0f), y3 = fmaxf(v[q * 8 + 3] + b0.w, 0.0f);
        const float y4 = fmaxf(v[q * 8 + 4] + b1.x, 0.0f), y5 = fmaxf(v[q * 8 + 5] + b1.y, 0.0f);
        const float y6 = fmaxf(v[q * 8 + 6] + b1.z, 0.0f), y7 = fmaxf(v[q * 8 + 7] + b1.w, 0.0f);
        st_shared_v4(dst + sw128_offset(row, k0 + q * 8, BM), pack2(y0, y1), pack2(y2, y3), pack2(y4, y5),
                     pack2(y6, y7));
    }
}

__device__ __forceinline__ void sync_for_mma() {
    fence_async_shared();      // generic-proxy writes of operands -> visible to the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// K-loop of one MMA chain: D[128 x N] (+)= A[128 x K] * B[N x K]^T, both
// operands K-major 128B-swizzled with panels of 64 K.
__device__ __forceinline__ void mma_chain(uint32_t d, uint32_t a_base, int a_rows, uint32_t b_base, int b_rows,
                                          int K, uint32_t idesc) {
    for (int kk = 0; kk < K / 16; ++kk) {
        const int panel = kk >> 2, sub = kk & 3;
        const uint64_t ad = sw128_desc(a_base + panel * (a_rows / 8) * 1024 + sub * 32);
        const uint64_t bd = sw128_desc(b_base + panel * (b_rows / 8) * 1024 + sub * 32);
        mma_bf16(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
    }
}

// Waits for the tensor core and agrees across the CTA on success.
__device__ __forceinline__ bool wait_mma(uint64_t* bar, uint32_t& phase) {
    // one warp polls the mbarrier; the others block in the barrier (issuing nothing),
    // which then carries the completion to them
    bool ok = true;
    if (threadIdx.x < 32) ok = mbar_wait(bar, phase);
    phase ^= 1;
    const bool all = __syncthreads_and(ok);
    tc_fence_after();
    return all;
}

__global__ void __launch_bounds__(BT, 1) policy_bf16_kernel(PolicyArgs a) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int row_in_tile = quarter * 32 + lane;     // TMEM lane of this thread
    const int H = a.H, O = a.O, I = a.in_dim;
    const BfLayout L = bf_layout(H, O);
    const NetOffsets off = net_offsets(I, H, O);
    const int ldo = O | 1;
    float* bias = (float*)(smem + L.bias);           // [b1 | c1 | b2 | c2 | b3 | c3]

    // weights -> shared memory, BF16, K-major (row n of B = output unit n): the
    // actor of w and the critic of wc (per-agent networks: packed again
    // whenever a tile's agent differs from the last one's)
    auto pack_weights = [&](const float* w, const float* wc) {
        pack_operand(smem + L.w1, 2 * H, KX, [&](int n, int k) {
            if (k >= I) return 0.0f;
            return n < H ? __ldg(w + off.W1 + (size_t)k * H + n) : __ldg(wc + off.V1 + (size_t)k * H + (n - H));
        });
        pack_operand(smem + L.w2a, H, H, [&](int n, int k) { return __ldg(w + off.W2 + (size_t)k * H + n); });
        pack_operand(smem + L.w2c, H, H, [&](int n, int k) { return __ldg(wc + off.V2 + (size_t)k * H + n); });
        pack_operand(smem + L.w3, L.N3, H, [&](int n, int k) {
            return n < O ? __ldg(w + off.W3 + (size_t)k * O + n) : 0.0f;
        });
        pack_operand(smem + L.v3, 16, H, [&](int n, int k) { return n == 0 ? __ldg(wc + off.V3 + k) : 0.0f; });
        for (int k = tid; k < 4 * H + O + 1; k += BT) {
            float v;
            if (k < H) v = w[off.b1 + k];
            else if (k < 2 * H) v = wc[off.c1 + k - H];
            else if (k < 3 * H) v = w[off.b2 + k - 2 * H];
            else if (k < 4 * H) v = wc[off.c2 + k - 3 * H];
            else if (k < 4 * H + O) v = w[off.b3 + k - 4 * H];
            else v = wc[off.c3];
            bias[k] = v;
        }
    };
    pack_weights(a.weights, a.weights);
    int packed = 0;                                  // agent whose weights are packed
    // padding columns of the observation operand stay zero for every tile
    for (int k = tid; k < BM * KX * 2 / 16; k += BT) st_shared_v4(smem + L.x + k * 16, 0u, 0u, 0u, 0u);
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, TMEM_COLS);
    sync_for_mma();
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t sx = smem_u32(smem + L.x), sh = smem_u32(smem + L.h);
    const uint32_t sw1 = smem_u32(smem + L.w1), sw2a = smem_u32(smem + L.w2a), sw2c = smem_u32(smem + L.w2c);
    const uint32_t sw3 = smem_u32(smem + L.w3), sv3 = smem_u32(smem + L.v3);
    float* stage = (float*)(smem + L.h);             // logits [BM][ldo], then sampler scratch [BM][ldo]
    float* wscr = (2 * ldo <= H) ? stage + BM * ldo : nullptr;   // scratch only if both fit the region
    float* vals = (float*)(smem + L.vals);
    uint32_t phase = 0;
    bool ok = true;
    // shared networks: tiles of BM consecutive rows, round robin over the CTAs;
    // per-agent networks: tiles of one agent over BM consecutive environments,
    // a contiguous range of them per CTA (agent-major, so a CTA meets few agents)
    const int n_env = a.rows / a.per_env;
    const int tpa = (n_env + BM - 1) / BM;
    const int n_tiles = a.agents ? a.agents * tpa : (a.rows + BM - 1) / BM;
    const int t_lo = a.agents ? (int)((long long)n_tiles * blockIdx.x / gridDim.x) : (int)blockIdx.x;
    const int t_hi = a.agents ? (int)((long long)n_tiles * (blockIdx.x + 1) / gridDim.x) : n_tiles;
    const int t_step = a.agents ? 1 : (int)gridDim.x;
    for (int tile = t_lo; tile < t_hi; tile += t_step) {
        const int agent = a.agents ? tile / tpa : 0;
        const int e0 = a.agents ? (tile % tpa) * BM : 0;
        const int row0 = a.agents ? 0 : tile * BM;
        const int nrows = a.agents ? min(BM, n_env - e0) : min(BM, a.rows - row0);
        auto row_of = [&](int r) { return a.agents ? (e0 + r) * a.per_env + agent : row0 + r; };
        if (a.agents && agent != packed) {
            __syncthreads();                             // the previous tile's MMAs are complete (waited)
            pack_weights(a.weights + (size_t)agent * a.actor_stride, a.weights + (size_t)agent * a.critic_stride);
            packed = agent;
        }
        // observations -> BF16 operand [BM][KX]: coalesced over the tile's contiguous rows, or
        // gathered row by row (per-agent tiles)
        if (!a.agents) {
            const float* src = a.x + (size_t)row0 * I;
            const int n = nrows * I;
            for (int idx = tid; idx < n; idx += BT) {
                const int r = idx / I, k = idx - r * I;
                const __nv_bfloat16 v = __float2bfloat16_rn(__ldg(src + idx));
                *reinterpret_cast<__nv_bfloat16*>(smem + L.x + sw128_offset(r, k, BM)) = v;
            }
        } else {
            for (int idx = tid; idx < BM * I; idx += BT) {
                const int r = idx / I, k = idx - r * I;
                const float f = r < nrows ? __ldg(a.x + (size_t)row_of(r) * I + k) : 0.0f;
                *reinterpret_cast<__nv_bfloat16*>(smem + L.x + sw128_offset(r, k, BM)) = __float2bfloat16_rn(f);
            }
        }
        sync_for_mma();
        // layer 1 of actor and critic: D[:, 0:2H] = X W1cat
        if (tid == 0) {
            mma_chain(tmem, sx, BM, sw1, 2 * H, KX, idesc_bf16(BM, 2 * H));
            mma_commit(&bar);
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        for (int c = 0; c < H / 32; ++c) {           // this warpgroup: actor (half 0) or critic (half 1)
            const int col = half * H + c * 32;
            epilogue32(lane_base + col, bias + col, smem + L.h, row_in_tile, col);
        }
        sync_for_mma();
        // layer 2: D[:, 0:H] = H1a W2, D[:, H:2H] = H1c V2
        if (tid == 0) {
            mma_chain(tmem, sh, BM, sw2a, H, H, idesc_bf16(BM, H));
            mma_chain(tmem + H, sh + (H / 64) * (BM / 8) * 1024, BM, sw2c, H, H, idesc_bf16(BM, H));
            mma_commit(&bar);
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        for (int c = 0; c < H / 32; ++c) {
            const int col = half * H + c * 32;
            epilogue32(lane_base + col, bias + 2 * H + col, smem + L.h, row_in_tile, col);
        }
        sync_for_mma();
        // heads: logits = H2a W3 (N3 columns), value = H2c V3 (column 0 of 16)
        if (tid == 0) {
            mma_chain(tmem + COL_D3, sh, BM, sw3, L.N3, H, idesc_bf16(BM, L.N3));
            mma_chain(tmem + COL_D4, sh + (H / 64) * (BM / 8) * 1024, BM, sv3, 16, H, idesc_bf16(BM, 16));
            mma_commit(&bar);
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        float* lrow = stage + row_in_tile * ldo;
        if (half == 0) {
            for (int c = 0; c * 32 < L.N3; ++c) {
                float v[32];
                tmem_ld32(lane_base + COL_D3 + c * 32, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = c * 32 + j;
                    if (col < O) lrow[col] = v[j] + bias[4 * H + col];
                }
            }
        } else {
            float vv[32];
            tmem_ld32(lane_base + COL_D4, vv);
            vals[row_in_tile] = vv[0] + bias[4 * H + O];
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (half == 0 && row_in_tile < nrows)
            sample_row(a, row_of(row_in_tile), lrow, vals[row_in_tile], wscr ? wscr + row_in_tile * ldo : nullptr);
        __syncthreads();
    }
    if (!ok) {
        // a wait gave up: give the tensor core one more bounded chance to finish before freeing TMEM
        mbar_wait(&bar, phase, 200000000LL);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Fast path for up to 64 logits and 32 inputs: the next tile's observations
// are loaded (coalesced 16-byte loads of the tile's contiguous rows) into
// registers while the current tile runs; ReLU epilogues on BF16 pairs; the
// sampler reads the logits from registers (same operations, same order as
// sample_head, so the drawn action is the same); the critic warpgroup writes
// the value.

template <int KT>
__device__ __forceinline__ int sample_head_reg(const float (&l)[KT], int lo, int K, uint32_t w0, uint32_t w1,
                                               float u, float& logp, float& ent) {
    auto ok = [&](int j) { return j >= lo && j < lo + K && ((((j < 32 ? w0 : w1) >> (j & 31)) & 1u) != 0); };
    float m = -FLT_MAX;
    bool any = false;
#pragma unroll
    for (int j = 0; j < KT; ++j)
        if (ok(j)) { any = true; m = fmaxf(m, l[j]); }
    if (!any) return -1;
    float S = 0.0f, dot = 0.0f;
    float wv[KT];
#pragma unroll
    for (int j = 0; j < KT; ++j) {
        wv[j] = -1.0f;
        if (ok(j)) {
            const float d = __fsub_rn(l[j], m);
            wv[j] = exp32(d);
            S = __fadd_rn(S, wv[j]);
            dot = fmaf(wv[j], d, dot);
        }
    }
    const float thr = __fmul_rn(u, S);
    float c = 0.0f, la = 0.0f, ll = 0.0f;
    int act = -1, last = -1;
#pragma unroll
    for (int j = 0; j < KT; ++j) {
        if (wv[j] >= 0.0f) {
            last = j;
            ll = l[j];
            c = __fadd_rn(c, wv[j]);
            if (act < 0 && c > thr) { act = j; la = l[j]; }
        }
    }
    if (act < 0) { act = last; la = ll; }
    const float logS = logf(S);
    logp += (la - m) - logS;
    ent += logS - dot / S;
    return act - lo;
}

template <int KT>
__global__ void __launch_bounds__(BT, 1) policy_bf16_fast_kernel(PolicyArgs a) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int row_in_tile = quarter * 32 + lane;
    const int H = a.H, O = a.O, I = a.in_dim;
    const BfLayout L = bf_layout(H, O);
    const NetOffsets off = net_offsets(I, H, O);
    const float* w = a.weights;

    pack_operand(smem + L.w1, 2 * H, KX, [&](int n, int k) {
        if (k >= I) return 0.0f;
        return n < H ? __ldg(w + off.W1 + (size_t)k * H + n) : __ldg(w + off.V1 + (size_t)k * H + (n - H));
    });
    pack_operand(smem + L.w2a, H, H, [&](int n, int k) { return __ldg(w + off.W2 + (size_t)k * H + n); });
    pack_operand(smem + L.w2c, H, H, [&](int n, int k) { return __ldg(w + off.V2 + (size_t)k * H + n); });
    pack_operand(smem + L.w3, L.N3, H, [&](int n, int k) {
        return n < O ? __ldg(w + off.W3 + (size_t)k * O + n) : 0.0f;
    });
    pack_operand(smem + L.v3, 16, H, [&](int n, int k) { return n == 0 ? __ldg(w + off.V3 + k) : 0.0f; });
    float* bias = (float*)(smem + L.bias);
    for (int k = tid; k < 4 * H + O + 1; k += BT) {
        float v;
        if (k < H) v = w[off.b1 + k];
        else if (k < 2 * H) v = w[off.c1 + k - H];
        else if (k < 3 * H) v = w[off.b2 + k - 2 * H];
        else if (k < 4 * H) v = w[off.c2 + k - 3 * H];
        else if (k < 4 * H + O) v = w[off.b3 + k - 4 * H];
        else v = w[off.c3];
        bias[k] = v;
    }
    for (int k = tid; k < BM * KX * 2 / 16; k += BT) st_shared_v4(smem + L.x + k * 16, 0u, 0u, 0u, 0u);
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, TMEM_COLS);
    sync_for_mma();
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t sx = smem_u32(smem + L.x), sh = smem_u32(smem + L.h);
    const uint32_t sw1 = smem_u32(smem + L.w1), sw2a = smem_u32(smem + L.w2a), sw2c = smem_u32(smem + L.w2c);
    const uint32_t sw3 = smem_u32(smem + L.w3), sv3 = smem_u32(smem + L.v3);
    const __nv_bfloat162 zero2 = __floats2bfloat162_rn(0.0f, 0.0f);

    // observations of a tile: its rows are contiguous; 4 float4 slots per thread
    float4 xr[4];
    auto load_obs = [&](int tile) {
        const int row0 = tile * BM;
        const int n = tile < (a.rows + BM - 1) / BM ? min(BM, a.rows - row0) * I : 0;
        const float* src = a.x + (size_t)row0 * I;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int f = (tid + q * BT) * 4;
            if (f + 3 < n) {
                xr[q] = __ldg(reinterpret_cast<const float4*>(src + f));
            } else {
                xr[q].x = f < n ? __ldg(src + f) : 0.0f;
                xr[q].y = f + 1 < n ? __ldg(src + f + 1) : 0.0f;
                xr[q].z = f + 2 < n ? __ldg(src + f + 2) : 0.0f;
                xr[q].w = f + 3 < n ? __ldg(src + f + 3) : 0.0f;
            }
        }
    };
    auto store_obs = [&]() {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int f = (tid + q * BT) * 4;
            if (f < BM * I) {
                int r = f / I, c = f - r * I;
                const float v[4] = {xr[q].x, xr[q].y, xr[q].z, xr[q].w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (r < BM)
                        *reinterpret_cast<__nv_bfloat16*>(smem + L.x + sw128_offset(r, c, BM)) = __float2bfloat16_rn(v[j]);
                    if (++c == I) { c = 0; ++r; }
                }
            }
        }
    };

    uint32_t phase = 0;
    bool ok = true;
    const int n_tiles = (a.rows + BM - 1) / BM;
    if ((int)blockIdx.x < n_tiles) load_obs(blockIdx.x);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int row0 = tile * BM;
        const int nrows = min(BM, a.rows - row0);
        store_obs();
        // this thread's row: sampling inputs, loaded early
        const int grow = row0 + row_in_tile;
        const bool live = row_in_tile < nrows;
        uint32_t w0 = 0xFFFFFFFFu, w1 = 0xFFFFFFFFu;
        float us[EJ_MAX_NB] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (half == 0 && live && a.act) {
            if (a.W) {
                const uint32_t* mw = a.mask + (size_t)grow * a.W;
                w0 = mw[0];
                w1 = (KT > 32 && a.W > 1) ? mw[1] : 0u;
            }
            if (a.u) {
#pragma unroll
                for (int h = 0; h < EJ_MAX_NB; ++h)
                    if (h < a.n_heads) us[h] = a.u[(size_t)grow * a.n_heads + h];
            } else {
                const int e = a.env0 + grow / a.per_env, i = grow % a.per_env;
                const uint4 x = philox4x32_10(make_uint4(a.stream_id == 0 ? (uint32_t)i : 0u, (uint32_t)e, a.gstep[e],
                                                         (uint32_t)a.stream_id), a.key[0], a.key[1]);
                if (a.stream_id == 0) us[0] = u01(x.w);
                else { us[0] = u01(x.x); us[1] = u01(x.y); us[2] = u01(x.z); us[3] = u01(x.w); }
            }
        }
        sync_for_mma();
        if (tid == 0) {
            mma_chain(tmem, sx, BM, sw1, 2 * H, KX, idesc_bf16(BM, 2 * H));
            mma_commit(&bar);
        }
        if (tile + (int)gridDim.x < n_tiles) load_obs(tile + gridDim.x);   // next tile, into registers
        if (!(ok = wait_mma(&bar, phase))) break;
        // layer-1 epilogue: this warpgroup's network (half 0 actor, half 1 critic), bias + ReLU on BF16 pairs
        for (int c = 0; c < H / 32; ++c) {
            const int col = half * H + c * 32;
            float v[32];
            tmem_ld32(lane_base + col, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t pk[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = q * 8 + 2 * j;
                    const __nv_bfloat162 y = __hmax2(__floats2bfloat162_rn(v[k] + bias[col + k], v[k + 1] + bias[col + k + 1]), zero2);
                    pk[j] = *reinterpret_cast<const uint32_t*>(&y);
                }
                st_shared_v4(smem + L.h + sw128_offset(row_in_tile, col + q * 8, BM), pk[0], pk[1], pk[2], pk[3]);
            }
        }
        sync_for_mma();
        if (tid == 0) {
            mma_chain(tmem, sh, BM, sw2a, H, H, idesc_bf16(BM, H));
            mma_chain(tmem + H, sh + (H / 64) * (BM / 8) * 1024, BM, sw2c, H, H, idesc_bf16(BM, H));
            mma_commit(&bar);
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        for (int c = 0; c < H / 32; ++c) {
            const int col = half * H + c * 32;
            float v[32];
            tmem_ld32(lane_base + col, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t pk[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = q * 8 + 2 * j;
                    const __nv_bfloat162 y = __hmax2(__floats2bfloat162_rn(v[k] + bias[2 * H + col + k],
                                                                           v[k + 1] + bias[2 * H + col + k + 1]), zero2);
                    pk[j] = *reinterpret_cast<const uint32_t*>(&y);
                }
                st_shared_v4(smem + L.h + sw128_offset(row_in_tile, col + q * 8, BM), pk[0], pk[1], pk[2], pk[3]);
            }
        }
        sync_for_mma();
        if (tid == 0) {
            mma_chain(tmem + COL_D3, sh, BM, sw3, L.N3, H, idesc_bf16(BM, L.N3));
            mma_chain(tmem + COL_D4, sh + (H / 64) * (BM / 8) * 1024, BM, sv3, 16, H, idesc_bf16(BM, 16));
            mma_commit(&bar);
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        if (half == 0) {
            float l[KT];
            {
                float v[32];
                tmem_ld32(lane_base + COL_D3, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) l[j] = v[j];
                if constexpr (KT == 64) {
                    tmem_ld32(lane_base + COL_D3 + 32, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) l[32 + j] = v[j];
                }
            }
#pragma unroll
            for (int j = 0; j < KT; ++j) l[j] = j < O ? l[j] + bias[4 * H + j] : 0.0f;
            if (live) {
                if (a.logits) {
#pragma unroll
                    for (int j = 0; j < KT; ++j)
                        if (j < O) a.logits[(size_t)grow * O + j] = l[j];
                }
                if (a.act) {
                    float logp = 0.0f, ent = 0.0f;
                    bool none = false;
                    for (int h = 0; h < a.n_heads; ++h) {
                        const float uh = h == 0 ? us[0] : h == 1 ? us[1] : h == 2 ? us[2] : us[3];
                        int act = sample_head_reg<KT>(l, h * a.head, a.head, w0, w1, uh, logp, ent);
                        if (act < 0) { act = 0; none = true; }
                        a.act[(size_t)grow * a.n_heads + h] = act;
                    }
                    if (none) { logp = 0.0f; ent = 0.0f; }
                    a.logp[grow] = logp;
                    if (a.entropy) a.entropy[grow] = ent;
                }
            }
        } else {
            // tcgen05.ld is warp-collective: every lane loads, live rows store
            float vv[32];
            tmem_ld32(lane_base + COL_D4, vv);
            if (live) a.value[grow] = vv[0] + bias[4 * H + O];
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (!ok) mbar_wait(&bar, phase, 200000000LL);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Several tile pipelines per CTA.  Actor and critic run in different CTAs
// (the sampler needs only the actor; the value is only written out), which
// halves the weights a CTA holds; each of its warpgroups then runs its own
// sequence of 128-row tiles with its own observation and activation buffers,
// its own TMEM columns and its own mbarrier, synchronising only through a
// named barrier of its 128 threads.  While one warpgroup runs an epilogue or
// the sampler, the tensor core runs the others' products.

// ---------------------------------------------------------------------------
// Pipelined kernel for hidden 128, up to 96 logits and 32 inputs, several
// networks per launch.  PP_NWG warpgroups per CTA, each an independent tile
// pipeline with its own observation and hidden operands in shared memory and
// its own 128 TMEM columns, which hold the layer products and then the head.
// Each CTA serves one network in one role (actor or critic): it packs that
// network's weights once and then takes that network's tiles PP_NWG at a time.

constexpr int PP_NWG = 4;       // tile pipelines per CTA
constexpr int PP_MAX_O = 96;    // logits: the head operand [N3][H] fits beside four pipelines
constexpr int PP_SCR = 64;      // exp weights a thread keeps in shared memory per head
// Cost of a tile in thousands of SM cycles, measured with clock64 stamps per
// phase on GB300 (hidden 128, three pipelines per CTA): the critic's tile
// about 12 (observations, three products, two epilogues, value); the actor's
// about 13 plus 2.2 per group of 8 logit columns its heads scan (24 logits:
// 7.1, 84 logits: 23.5).
constexpr double PP_CRITIC_TILE = 12.0, PP_ACTOR_TILE = 13.0, PP_ACTOR_GROUP = 2.2;

struct PpLayout {
    uint32_t w1, w2, w3, h[PP_NWG], bias, total;
};

__host__ __device__ inline PpLayout pp_layout(int H, int n3_max) {
    PpLayout L;
    uint32_t b = 0;
    L.w1 = b; b += (uint32_t)H * KX * 2;                        // [H][KX]
    L.w2 = b; b += (uint32_t)H * H * 2;                         // [H][H]
    L.w3 = b; b += (uint32_t)(n3_max > 16 ? n3_max : 16) * H * 2;   // [N3][H] (actor) or [16][H] (critic)
    // a pipeline's observation operand [BM][K1 <= 32] is the second 64-column
    // panel of its hidden operand: free from the tile's start until the
    // layer-1 product has read it (the first panel stages the floats)
    for (int w = 0; w < PP_NWG; ++w) { L.h[w] = b; b += (uint32_t)BM * H * 2; }
    L.bias = b; b += ((2u * H + (uint32_t)n3_max + 4) * 4 + 1023) & ~1023u;   // layer 1 | layer 2 | head (to N3)
    L.total = b;
    return L;
}

// Two float32 additions in one instruction (add.rn.f32x2: each rounded once,
// as two scalar additions), and two floats -> BF16 pair with negatives set
// to 0 (cvt.rn.relu: ReLU then round, the same values as round then ReLU).
__device__ __forceinline__ void add2_rn(float& a, float& b, float c, float d) {
    unsigned long long x, y, z;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a), "f"(b));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(c), "f"(d));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(z));
}
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ unsigned long long f2(float a, float b) {
    unsigned long long x;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a), "f"(b));
    return x;
}
__device__ __forceinline__ void f2_split(unsigned long long x, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
}
__device__ __forceinline__ unsigned long long mul2_rn(unsigned long long x, unsigned long long y) {
    unsigned long long z;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
    return z;
}
__device__ __forceinline__ unsigned long long sub2_rn(unsigned long long x, unsigned long long y) {
    unsigned long long z;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
    return z;
}
__device__ __forceinline__ unsigned long long fadd2_rn(unsigned long long x, unsigned long long y) {
    unsigned long long z;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(y));
    return z;
}

// exp32 of two arguments at once: exp32's operations in exp32's order, the
// float32 ones on pairs (f32x2 arithmetic rounds each element once, as the
// scalar operation does), so each result equals exp32 of its argument.
__device__ __forceinline__ void exp32x2(float xa, float xb, float& ea, float& eb) {
    auto c2 = [](float c) { return f2(c, c); };
    const unsigned long long X = f2(xa, xb);
    float na, nb;
    f2_split(mul2_rn(X, c2(0x1.715476p+0f)), na, nb);
    na = rintf(na);
    nb = rintf(nb);
    const unsigned long long N = f2(na, nb);
    unsigned long long R = sub2_rn(X, mul2_rn(N, c2(0x1.62e4p-1f)));
    R = sub2_rn(R, mul2_rn(N, c2(0x1.7f7d1cp-20f)));
    unsigned long long P = c2(0x1.a01a02p-13f);
    P = fadd2_rn(mul2_rn(P, R), c2(0x1.6c16c2p-10f));
    P = fadd2_rn(mul2_rn(P, R), c2(0x1.111112p-7f));
    P = fadd2_rn(mul2_rn(P, R), c2(0x1.555556p-5f));
    P = fadd2_rn(mul2_rn(P, R), c2(0x1.555556p-3f));
    P = fadd2_rn(mul2_rn(P, R), c2(0.5f));
    P = fadd2_rn(mul2_rn(P, R), c2(1.0f));
    P = fadd2_rn(mul2_rn(P, R), c2(1.0f));
    const unsigned long long S = f2(__int_as_float(((int)na + 127) << 23), __int_as_float(((int)nb + 127) << 23));
    f2_split(mul2_rn(P, S), ea, eb);
    ea = xa < -80.0f ? 0.0f : ea;
    eb = xb < -80.0f ? 0.0f : eb;
}

__device__ __forceinline__ void wg_bar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

__device__ __forceinline__ bool wg_and(int id, bool v) {
    uint32_t out;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n barrier.red.and.pred p, %2, 128, p;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(out)
        : "r"((uint32_t)v), "r"(id)
        : "memory");
    return out != 0;
}

__device__ __forceinline__ void wg_sync_for_mma(int id) {
    fence_async_shared();
    tc_fence_before();
    wg_bar(id);
    tc_fence_after();
}

__device__ __forceinline__ bool wg_wait_mma(uint64_t* bar, uint32_t& phase, int id) {
    bool ok = true;
    if ((threadIdx.x & 127) < 32) ok = mbar_wait(bar, phase);   // the warpgroup's first warp polls
    phase ^= 1;
    const bool all = wg_and(id, ok);
    tc_fence_after();
    return all;
}

// The inverse-CDF draw of one head: logits = this lane's TMEM columns
// [lo, lo + K) + the head bias b3, under the mask words mw.  Same operations
// in the same order as sample_head, so the draw is the same.  Each pass walks
// the head in groups of 8 columns (one 8-column TMEM load each) in a loop
// that is not unrolled: the sampler runs once per row and tile, and a long
// unrolled body would be fetched from L2 every time.  Every step within a
// group is a select on the column's valid bit (the lanes' masks differ).  The
// exp weights of the first PP_SCR columns are kept in scr (this thread's
// column of a [PP_SCR][128] float array), the others are recomputed.  lo and
// K are warp-uniform (every lane loads).  Returns the action (-1: nothing
// allowed) and adds the head's log probability and entropy.
__device__ __forceinline__ uint32_t group_bits(const uint32_t (&mw)[4], int g, int lo, int hi) {
    const int c = g >> 5;
    const uint32_t wd = c == 0 ? mw[0] : c == 1 ? mw[1] : c == 2 ? mw[2] : mw[3];
    uint32_t b = (wd >> (g & 31)) & 0xFFu;                  // mask bits of columns g .. g + 7
    if (lo > g) b &= 0xFFu << (lo - g);                     // lo - g < 8: g starts at lo rounded down
    if (hi - g < 8) b &= (1u << (hi - g)) - 1u;
    return b;
}

__device__ __forceinline__ int sample_head_tmem(uint32_t taddr, const float* b3, int lo, int K, const uint32_t (&mw)[4],
                                             float u, float* scr, float& logp, float& ent) {
    const int g0 = lo & ~7, hi = lo + K;
    float m = -FLT_MAX;
    uint32_t any = 0;
#pragma unroll 1
    for (int g = g0; g < hi; g += 8) {
        float v[8];
        tmem_ld8(taddr + (uint32_t)g, v);
        const uint32_t vb = group_bits(mw, g, lo, hi);
        any |= vb;
#pragma unroll
        for (int j = 0; j < 8; ++j) m = ((vb >> j) & 1u) ? fmaxf(m, v[j] + b3[g + j]) : m;
    }
    float S = 0.0f, dot = 0.0f;
#pragma unroll 1
    for (int g = g0; g < hi; g += 8) {
        float v[8];
        tmem_ld8(taddr + (uint32_t)g, v);
        const uint32_t vb = group_bits(mw, g, lo, hi);
        float d[8], wv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) d[j] = ((vb >> j) & 1u) ? __fsub_rn(v[j] + b3[g + j], m) : 0.0f;
#pragma unroll
        for (int j = 0; j < 8; j += 2) exp32x2(d[j], d[j + 1], wv[j], wv[j + 1]);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool ok = (vb >> j) & 1u;
            S = ok ? __fadd_rn(S, wv[j]) : S;
            dot = ok ? fmaf(wv[j], d[j], dot) : dot;
            const int k = g + j - lo;
            if (ok && k < PP_SCR) scr[k * 128] = wv[j];
        }
    }
    const float thr = __fmul_rn(u, S);
    float cum = 0.0f, la = 0.0f, ll = 0.0f;
    int act = -1, last = -1;
#pragma unroll 1
    for (int g = g0; g < hi; g += 8) {
        float v[8];
        tmem_ld8(taddr + (uint32_t)g, v);
        const uint32_t vb = group_bits(mw, g, lo, hi);
        float wv[8];
        if (g + 7 - lo < PP_SCR) {            // uniform: the group's weights are in scr
#pragma unroll
            for (int j = 0; j < 8; ++j) wv[j] = scr[(((vb >> j) & 1u) ? g + j - lo : 0) * 128];
        } else {
            float d[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) d[j] = ((vb >> j) & 1u) ? __fsub_rn(v[j] + b3[g + j], m) : 0.0f;
#pragma unroll
            for (int j = 0; j < 8; j += 2) exp32x2(d[j], d[j + 1], wv[j], wv[j + 1]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = g + j - lo;
                if (k < PP_SCR) wv[j] = scr[(k >= 0 ? k : 0) * 128];
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool ok = (vb >> j) & 1u;
            const float l = v[j] + b3[g + j];
            const float cn = __fadd_rn(cum, wv[j]);
            cum = ok ? cn : cum;
            const bool hit = ok && act < 0 && cn > thr;
            act = hit ? g + j : act;
            la = hit ? l : la;
            last = ok ? g + j : last;
            ll = ok ? l : ll;
        }
    }
    if (any == 0) return -1;
    if (act < 0) { act = last; la = ll; }
    const float logS = logf(S);
    logp += (la - m) - logS;
    ent += logS - dot / S;
    return act - lo;
}

__global__ void __launch_bounds__(128 * PP_NWG, 1) policy_bf16_pp_kernel(const __grid_constant__ PolicyLaunch pl) {
    constexpr int NWG = PP_NWG;
    constexpr int NTH = 128 * NWG;
    static_assert(NWG * 128 <= (int)TMEM_COLS, "TMEM columns");
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bars[NWG];
    __shared__ uint32_t tmem_slot;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wg = warp >> 2, quarter = warp & 3;
    const int wtid = tid & 127;
    const int row_in_tile = quarter * 32 + lane;     // TMEM lane of this thread (within its warpgroup)
    const int bar_id = 1 + wg;
    const int H = pl.H;
    const PpLayout L = pp_layout(H, pl.n3_max);
    // this CTA's network and role
    int ni = 0;
    while (ni + 1 < pl.n_net && (int)blockIdx.x >= pl.net[ni + 1].cta0) ++ni;
    const PolicyNet& nt = pl.net[ni];
    const int O = nt.O, I = nt.in_dim, N3 = (O + 15) / 16 * 16;
    const NetOffsets off = net_offsets(I, H, O);
    const float* w = nt.weights;
    const int local = (int)blockIdx.x - nt.cta0;
    const bool actor = local < nt.n_act;
    const int role_cta = actor ? local : local - nt.n_act;
    const int role_ctas = actor ? nt.n_act : nt.n_cri;

    const size_t oW1 = actor ? off.W1 : off.V1, oW2 = actor ? off.W2 : off.V2;
    pack_operand(smem + L.w1, H, KX, [&](int n, int k) { return k < I ? __ldg(w + oW1 + (size_t)k * H + n) : 0.0f; });
    pack_operand(smem + L.w2, H, H, [&](int n, int k) { return __ldg(w + oW2 + (size_t)k * H + n); });
    if (actor)
        pack_operand(smem + L.w3, N3, H, [&](int n, int k) { return n < O ? __ldg(w + off.W3 + (size_t)k * O + n) : 0.0f; });
    else
        pack_operand(smem + L.w3, 16, H, [&](int n, int k) { return n == 0 ? __ldg(w + off.V3 + k) : 0.0f; });
    float* bias = (float*)(smem + L.bias);   // [0,H) layer 1, [H,2H) layer 2, [2H, 2H+N3) head (critic: 2H = c3)
    for (int k = tid; k < 2 * H + pl.n3_max; k += NTH) {
        float v = 0.0f;
        if (k < H) v = w[(actor ? off.b1 : off.c1) + k];
        else if (k < 2 * H) v = w[(actor ? off.b2 : off.c2) + k - H];
        else if (actor) v = k - 2 * H < O ? w[off.b3 + k - 2 * H] : 0.0f;
        else v = k == 2 * H ? w[off.c3] : 0.0f;
        bias[k] = v;
    }
    if (tid == 0) {
        for (int q = 0; q < NWG; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, TMEM_COLS);
    sync_for_mma();
    const uint32_t tcol = tmem_slot + (uint32_t)wg * 128u;                   // this pipeline's columns
    const uint32_t lane_base = tcol + ((uint32_t)(quarter * 32) << 16);
    uint8_t* hb = smem + L.h[wg];
    uint8_t* xb = hb + BM * 64 * 2;                     // the hidden operand's second panel
    const int K1 = (I + 15) & ~15;                      // layer-1 K: the inputs rounded up to an MMA step
    float* scr = reinterpret_cast<float*>(hb) + wtid;   // sampler scratch: the hidden operand is free after layer 3
    const uint32_t sx = smem_u32(xb), sh = smem_u32(hb);
    const uint32_t sw1 = smem_u32(smem + L.w1), sw2 = smem_u32(smem + L.w2), sw3 = smem_u32(smem + L.w3);
    uint64_t* bar = &bars[wg];

    // a tile's observations (contiguous rows, n = rows x I floats from src):
    // 8 float4 slots per thread of the warpgroup, slot q holding the floats
    // [f - mis, f - mis + 4) of the tile, f = (wtid + 128 q) * 4, where src is
    // mis floats past a 16-byte boundary; 16-byte loads where the 4 floats are
    // all in the tile, single loads at its ends (nothing outside it is read)
    constexpr int XS = 8;
    float4 xr[XS];
    int mis = 0;
    const int n_tiles = nt.n_tiles;
    auto seg_of = [&](int tile) {
        int q = nt.seg_lo;
        while (q + 1 < nt.seg_hi && tile >= pl.seg[q + 1].tile0) ++q;
        return q;
    };
    auto load_obs = [&](int tile) {
        const PolicySeg& sg = pl.seg[tile < n_tiles ? seg_of(tile) : nt.seg_lo];
        const int row0 = (tile - sg.tile0) * BM;
        const int n = tile < n_tiles ? min(BM, sg.rows - row0) * I : 0;
        const float* src = sg.x + (size_t)(n > 0 ? row0 : 0) * I;
        mis = (int)(((uintptr_t)src & 15) >> 2);
#pragma unroll
        for (int q = 0; q < XS; ++q) {
            const int r0 = (wtid + q * 128) * 4 - mis;
            if (r0 >= 0 && r0 + 3 < n) {
                xr[q] = __ldg(reinterpret_cast<const float4*>(src + r0));
            } else {
                xr[q].x = r0 >= 0 && r0 < n ? __ldg(src + r0) : 0.0f;
                xr[q].y = r0 + 1 >= 0 && r0 + 1 < n ? __ldg(src + r0 + 1) : 0.0f;
                xr[q].z = r0 + 2 >= 0 && r0 + 2 < n ? __ldg(src + r0 + 2) : 0.0f;
                xr[q].w = r0 + 3 < n ? __ldg(src + r0 + 3) : 0.0f;
            }
        }
    };
    // observations -> BF16 operand: the prefetched floats go row-major into the
    // hidden operand's first panel (free at the start of a tile), then each
    // thread converts its own row in 16-byte chunks up to K1 (columns I.. are
    // zero) into the second panel
    auto store_obs = [&]() {
        float* stage = reinterpret_cast<float*>(hb);
        wg_bar(bar_id);                        // every warp is done with the last tile's sampler scratch
#pragma unroll
        for (int q = 0; q < XS; ++q) {
            const int r0 = (wtid + q * 128) * 4 - mis;
            if (mis == 0) {
                if (r0 < BM * I) *reinterpret_cast<float4*>(stage + r0) = xr[q];
            } else {
                if (r0 >= 0 && r0 < BM * I) stage[r0] = xr[q].x;
                if (r0 + 1 >= 0 && r0 + 1 < BM * I) stage[r0 + 1] = xr[q].y;
                if (r0 + 2 >= 0 && r0 + 2 < BM * I) stage[r0 + 2] = xr[q].z;
                if (r0 + 3 < BM * I) stage[r0 + 3] = xr[q].w;
            }
        }
        wg_bar(bar_id);
        const float* srow = stage + row_in_tile * I;
#pragma unroll 1
        for (int c8 = 0; c8 < K1; c8 += 8) {
            float f8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) f8[j] = c8 + j < I ? srow[c8 + j] : 0.0f;
            st_shared_v4(xb + sw128_offset(row_in_tile, c8, BM), pack2(f8[0], f8[1]), pack2(f8[2], f8[3]),
                         pack2(f8[4], f8[5]), pack2(f8[6], f8[7]));
        }
    };
    auto relu_epi = [&](int bias_off) {
        for (int c = 0; c < H / 32; ++c) {
            float v[32];
            tmem_ld32(lane_base + c * 32, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 b0 = *reinterpret_cast<const float4*>(bias + bias_off + c * 32 + q * 8);
                const float4 b1 = *reinterpret_cast<const float4*>(bias + bias_off + c * 32 + q * 8 + 4);
                float* y = v + q * 8;
                add2_rn(y[0], y[1], b0.x, b0.y);
                add2_rn(y[2], y[3], b0.z, b0.w);
                add2_rn(y[4], y[5], b1.x, b1.y);
                add2_rn(y[6], y[7], b1.z, b1.w);
                st_shared_v4(hb + sw128_offset(row_in_tile, c * 32 + q * 8, BM), relu_bf16x2(y[0], y[1]),
                             relu_bf16x2(y[2], y[3]), relu_bf16x2(y[4], y[5]), relu_bf16x2(y[6], y[7]));
            }
        }
    };

    uint32_t phase = 0;
    bool ok = true;
    const int first = role_cta * NWG + wg, stride = role_ctas * NWG;
    if (first < n_tiles) load_obs(first);
    for (int tile = first; tile < n_tiles; tile += stride) {
        const PolicySeg& sg = pl.seg[seg_of(tile)];
        const int row0 = (tile - sg.tile0) * BM;
        const int nrows = min(BM, sg.rows - row0);
        store_obs();
        const int grow = row0 + row_in_tile;
        const bool live = row_in_tile < nrows;
        wg_sync_for_mma(bar_id);
        if (wtid == 0) {
            mma_chain(tcol, sx, BM, sw1, H, K1, idesc_bf16(BM, H));
            mma_commit(bar);
        }
        // the sampler's mask words and uniforms: their loads overlap the products
        uint32_t mw[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
        float us[EJ_MAX_NB] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (actor && live && sg.act) {
            if (nt.W) {
                const uint32_t* m = sg.mask + (size_t)grow * nt.W;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < nt.W) mw[k] = m[k];
            }
            if (sg.u) {
#pragma unroll
                for (int h = 0; h < EJ_MAX_NB; ++h)
                    if (h < nt.n_heads) us[h] = sg.u[(size_t)grow * nt.n_heads + h];
            } else {
                const int e = sg.env0 + grow / sg.per_env, i = grow % sg.per_env;
                const uint4 x = philox4x32_10(make_uint4(nt.stream_id == 0 ? (uint32_t)i : 0u, (uint32_t)e,
                                                         sg.gstep[e], (uint32_t)nt.stream_id),
                                              sg.key[0], sg.key[1]);
                if (nt.stream_id == 0) us[0] = u01(x.w);
                else { us[0] = u01(x.x); us[1] = u01(x.y); us[2] = u01(x.z); us[3] = u01(x.w); }
            }
        }
        if (tile + stride < n_tiles) load_obs(tile + stride);
        if (!(ok = wg_wait_mma(bar, phase, bar_id))) break;
        relu_epi(0);
        wg_sync_for_mma(bar_id);
        if (wtid == 0) {
            mma_chain(tcol, sh, BM, sw2, H, H, idesc_bf16(BM, H));
            mma_commit(bar);
        }
        if (!(ok = wg_wait_mma(bar, phase, bar_id))) break;
        relu_epi(H);
        wg_sync_for_mma(bar_id);   // the layer-2 product has been read: the head goes to the same columns
        if (wtid == 0) {
            if (actor) mma_chain(tcol, sh, BM, sw3, N3, H, idesc_bf16(BM, N3));
            else mma_chain(tcol, sh, BM, sw3, 16, H, idesc_bf16(BM, 16));
            mma_commit(bar);
        }
        if (!(ok = wg_wait_mma(bar, phase, bar_id))) break;
        if (actor) {
            const float* b3 = bias + 2 * H;
            if (sg.logits) {
                for (int c = 0; c < (O + 31) / 32; ++c) {
                    float v[32];
                    tmem_ld32(lane_base + c * 32, v);       // warp-collective: every lane loads
                    if (live) {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (c * 32 + j < O) sg.logits[(size_t)grow * O + c * 32 + j] = v[j] + b3[c * 32 + j];
                    }
                }
            }
            if (sg.act) {
                float logp = 0.0f, ent = 0.0f;
                bool none = false;
                for (int h = 0; h < nt.n_heads; ++h) {
                    const float uh = h == 0 ? us[0] : h == 1 ? us[1] : h == 2 ? us[2] : us[3];
                    int act = sample_head_tmem(lane_base, b3, h * nt.head, nt.head, mw, uh, scr, logp, ent);
                    if (act < 0) { act = 0; none = true; }
                    if (live) sg.act[(size_t)grow * nt.n_heads + h] = act;
                }
                if (none) { logp = 0.0f; ent = 0.0f; }
                if (live) {
                    sg.logp[grow] = logp;
                    if (sg.entropy) sg.entropy[grow] = ent;
                }
            }
        } else {
            float vv[32];
            tmem_ld32(lane_base, vv);                // warp-collective: every lane loads
            if (live) sg.value[grow] = vv[0] + bias[2 * H];
        }
    }
    if (!ok) mbar_wait(bar, phase, 200000000LL);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem_slot, TMEM_COLS);
}

}  // namespace

size_t policy_bf16_smem(int H, int O) { return bf_layout(H, O).total + 1024; }

namespace {

bool pp_takes(const PolicyArgs& a) {
    // observations: 4-byte aligned (16-byte when a row is 32 floats: a tile's
    // 4096 floats then fill the eight 16-byte slots of every thread exactly)
    return a.H == 128 && a.O >= 1 && a.O <= PP_MAX_O && a.in_dim <= 32 && a.W <= 4 && a.n_heads >= 1 &&
           a.n_heads <= EJ_MAX_NB && a.head >= 1 && a.n_heads * a.head == a.O && a.rows >= 1 &&
           ((uintptr_t)a.x & 3) == 0 && (a.in_dim < 32 || ((uintptr_t)a.x & 15) == 0);
}

bool same_net(const PolicyArgs& a, const PolicyArgs& b) {
    return a.weights == b.weights && a.in_dim == b.in_dim && a.O == b.O && a.n_heads == b.n_heads &&
           a.head == b.head && a.W == b.W && a.stream_id == b.stream_id;
}

int sm_count() {
    const int n = device_sms();
    return n < 2 ? 2 : n;
}

}  // namespace

ej_status launch_policy_bf16_multi(const PolicyArgs* segs, int n, cudaStream_t stream, bool* handled) {
    *handled = false;
    if (n < 1 || n > EJ_MAX_SEG) return fail(EJ_ERR_ARG, "bf16 policy: 1 to %d segments", EJ_MAX_SEG);
    for (int q = 0; q < n; ++q)
        if (!pp_takes(segs[q]) || segs[q].H != segs[0].H) return EJ_OK;
    // networks in order of first appearance; their segments contiguous
    PolicyLaunch pl;
    memset(&pl, 0, sizeof pl);
    pl.H = segs[0].H;
    int rep[EJ_MAX_NET], net_of[EJ_MAX_SEG];
    int n_net = 0;
    for (int q = 0; q < n; ++q) {
        int k = 0;
        while (k < n_net && !same_net(segs[rep[k]], segs[q])) ++k;
        if (k == n_net) {
            if (n_net == EJ_MAX_NET) return EJ_OK;
            rep[n_net++] = q;
        }
        net_of[q] = k;
    }
    pl.n_net = n_net;
    pl.n_seg = n;
    int total_tiles = 0, q_out = 0;
    for (int k = 0; k < n_net; ++k) {
        const PolicyArgs& r = segs[rep[k]];
        PolicyNet& nt = pl.net[k];
        nt.weights = r.weights; nt.in_dim = r.in_dim; nt.O = r.O; nt.n_heads = r.n_heads; nt.head = r.head;
        nt.W = r.W; nt.stream_id = r.stream_id;
        nt.seg_lo = q_out;
        int tiles = 0;
        for (int q = 0; q < n; ++q) {
            if (net_of[q] != k) continue;
            const PolicyArgs& a = segs[q];
            PolicySeg& g = pl.seg[q_out++];
            g.x = a.x; g.mask = a.mask; g.u = a.u; g.gstep = a.gstep; g.key = a.key;
            g.act = a.act; g.logp = a.logp; g.value = a.value; g.entropy = a.entropy; g.logits = a.logits;
            g.rows = a.rows; g.per_env = a.per_env; g.tile0 = tiles; g.env0 = a.env0;
            tiles += (a.rows + BM - 1) / BM;
        }
        nt.seg_hi = q_out;
        nt.n_tiles = tiles;
        total_tiles += tiles;
        const int n3 = (r.O + 15) / 16 * 16;
        if (n3 > pl.n3_max) pl.n3_max = n3;
    }
    // CTAs: at most one per SM, split over the networks and roles.  A role
    // with n CTAs runs its tiles in ceil(tiles / (n PP_NWG)) rounds of its
    // tile cost; the split is the one with the smallest longest role time
    // (binary search over the candidate times cost x rounds).
    const int sms = sm_count();
    const int n_role = 2 * n_net;
    double cost[2 * EJ_MAX_NET];
    int tiles[2 * EJ_MAX_NET];
    for (int k = 0; k < n_net; ++k) {
        const PolicyNet& nt = pl.net[k];
        int groups = 0;
        for (int h = 0; h < nt.n_heads; ++h) {
            const int lo = h * nt.head, hi = lo + nt.head;
            groups += (hi + 7) / 8 - lo / 8;
        }
        cost[2 * k] = PP_ACTOR_TILE + PP_ACTOR_GROUP * groups;
        cost[2 * k + 1] = PP_CRITIC_TILE;
        tiles[2 * k] = tiles[2 * k + 1] = nt.n_tiles;
    }
    auto ctas_for = [&](int r, double T) {        // fewest CTAs of role r finishing within T (0: impossible)
        const int rounds = (int)(T / cost[r] + 1e-9);
        if (rounds < 1) return 0;
        const int per = rounds * PP_NWG;
        return (tiles[r] + per - 1) / per;
    };
    auto fits = [&](double T, int* n) {
        int sum = 0;
        for (int r = 0; r < n_role; ++r) {
            const int c = ctas_for(r, T);
            if (c == 0) return false;
            if (n) n[r] = c;
            sum += c;
        }
        return sum <= sms;
    };
    double lo_T = 0.0, hi_T = 0.0;
    for (int r = 0; r < n_role; ++r) {
        const double t1 = cost[r] * ((tiles[r] + PP_NWG - 1) / PP_NWG);   // one CTA per role
        if (t1 > hi_T) hi_T = t1;
    }
    int n_ctas[2 * EJ_MAX_NET];
    if (!fits(hi_T, n_ctas)) return fail(EJ_ERR_UNSUPPORTED, "bf16 policy: more roles than SMs");
    // the smallest feasible time is cost[r] x q for some role r and rounds q: bisect on the value, then snap
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo_T + hi_T);
        if (fits(mid, nullptr)) hi_T = mid;
        else lo_T = mid;
    }
    fits(hi_T, n_ctas);
    for (int k = 0; k < n_net; ++k) {
        pl.net[k].n_act = n_ctas[2 * k];
        pl.net[k].n_cri = n_ctas[2 * k + 1];
    }
    int cta = 0;
    for (int k = 0; k < n_net; ++k) {
        pl.net[k].cta0 = cta;
        cta += pl.net[k].n_act + pl.net[k].n_cri;
    }
    const size_t smem = pp_layout(pl.H, pl.n3_max).total + 1024;
    static SmemOptIn opt_in;
    ej_status st = opt_in.ensure((const void*)policy_bf16_pp_kernel, smem);
    if (st != EJ_OK) return st;
    *handled = true;
    policy_bf16_pp_kernel<<<cta, 128 * PP_NWG, smem, stream>>>(pl);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "bf16 policy launch: %s", cudaGetErrorString(err));
    return EJ_OK;
}

// ---------------------------------------------------------------------------
// Hidden 256 (Section 5's networks).  One network's weights in BF16 are
// 2 x 128 KB for W2 / V2 alone, more than a CTA's shared memory beside the
// operands, so two CTAs of a thread-block cluster share a tile: both compute
// layer 1 in full (W1 resident in each), CTA rank r computes output units
// [128 r, 128 r + 128) of layer 2 (its half of W2 resident) and the head's
// partial sum over those units (its half of W3, or of V3 as a dot product in
// the epilogue).  Rank 1 stores its partial logits (or values) into rank 0's
// shared memory (distributed shared memory) between two cluster barriers;
// rank 0 adds its own and the bias, puts the logits back into TMEM and
// samples them with the pipelined kernel's sampler.  Clusters are actor or critic
// clusters of one network (as the pipelined kernel's CTAs), persistent over
// 128-row tiles; per-agent networks take agent-major tile ranges and pack an
// agent's weights when the agent changes.
constexpr int WD_H = 256;           // hidden units of this kernel
constexpr int WD_HALF = WD_H / 2;   // layer-2 output units per CTA
constexpr int WD_MAX_O = 64;        // logits: the head's TMEM columns and the sampler's scratch
constexpr int WD_RECV = 64;         // floats per row of the partial logits received by rank 0

struct WdLayout {
    uint32_t w1, w2, w3, x, h, bias, total;
};

// w1 [256][KX], w2 [128][256] (this rank's output units), w3 [64][128] (head
// rows, this rank's input units), x [BM][KX], h [BM][256]; bias floats: b1 /
// c1 [256], b2 / c2 half [128], b3 [64], V3 half rounded to BF16 [128], c3.
__host__ __device__ inline WdLayout wd_layout() {
    WdLayout L;
    uint32_t b = 0;
    L.w1 = b; b += WD_H * KX * 2;
    L.w2 = b; b += WD_HALF * WD_H * 2;
    L.w3 = b; b += 64 * WD_HALF * 2;
    L.x = b;  b += BM * KX * 2;
    L.h = b;  b += BM * WD_H * 2;
    L.bias = b; b += (WD_H + WD_HALF + 64 + WD_HALF + 4) * 4;
    L.total = b;
    return L;
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of both CTAs of the cluster; releases this CTA's earlier
// shared-memory writes (local and remote) to the other's later reads.
__device__ __forceinline__ void cluster_sync() {
    __syncwarp();                                    // the .aligned form wants converged warps
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address in the CTA of rank `rank` of the same shared-memory offset as `local`.
__device__ __forceinline__ uint32_t cluster_addr(const void* local, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(local)), "r"(rank));
    return remote;
}
__device__ __forceinline__ void st_cluster_f32(const void* local, uint32_t rank, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(cluster_addr(local, rank)), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_v4(uint32_t remote, float a, float b, float c, float d) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(remote), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane <- v.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]),
        "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]),
        "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]),
        "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void st_shared_b32(uint8_t* p, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

// Sum over 32 accumulator columns of relu(acc + bias) rounded to BF16, times
// dot[k] (the critic's value head on this rank's units; nothing is stored).
__device__ __forceinline__ float dot32(uint32_t taddr, const float* bias, const float* dot) {
    float v[32];
    tmem_ld32(taddr, v);
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j)
        acc = fmaf(__bfloat162float(__float2bfloat16_rn(fmaxf(v[j] + bias[j], 0.0f))), dot[j], acc);
    return acc;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(BT, 1)
    policy_bf16_wide_kernel(PolicyArgs a, int n_act_pairs) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ float vpart[2][BM];     // critic: this rank's partial values, one per warpgroup
    __shared__ float vrecv[BM];        // critic rank 0: rank 1's partial values
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const WdLayout L = wd_layout();
    const uint32_t rank = cluster_rank();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;             // TMEM lane of this thread
    const int pair = (int)blockIdx.x / 2, n_pairs = (int)gridDim.x / 2;
    const bool actor = pair < n_act_pairs;
    const int role_pair = actor ? pair : pair - n_act_pairs;
    const int role_pairs = actor ? n_act_pairs : n_pairs - n_act_pairs;
    const int I = a.in_dim, O = a.O, N3 = (O + 15) & ~15;
    const NetOffsets off = net_offsets(I, WD_H, O);
    float* b1 = (float*)(smem + L.bias);             // [256] b1 | c1
    float* b2 = b1 + WD_H;                           // [128] b2 | c2 of this rank's units
    float* b3 = b2 + WD_HALF;                        // [64]
    float* v3r = b3 + 64;                            // [128] critic: V3 of this rank's units, BF16-rounded
    float* c3 = v3r + WD_HALF;
    const int u0 = (int)rank * WD_HALF;              // this rank's first layer-2 unit

    auto pack_weights = [&](const float* w) {
        const size_t o1 = actor ? off.W1 : off.V1, o2 = actor ? off.W2 : off.V2;
        pack_operand(smem + L.w1, WD_H, KX,
                     [&](int n, int k) { return k < I ? __ldg(w + o1 + (size_t)k * WD_H + n) : 0.0f; });
        pack_operand(smem + L.w2, WD_HALF, WD_H, [&](int n, int k) { return __ldg(w + o2 + (size_t)k * WD_H + u0 + n); });
        if (actor)
            pack_operand(smem + L.w3, 64, WD_HALF, [&](int n, int k) {
                return n < O ? __ldg(w + off.W3 + (size_t)(u0 + k) * O + n) : 0.0f;
            });
        for (int k = tid; k < WD_H; k += BT) b1[k] = w[(actor ? off.b1 : off.c1) + k];
        for (int k = tid; k < WD_HALF; k += BT) {
            b2[k] = w[(actor ? off.b2 : off.c2) + u0 + k];
            v3r[k] = actor ? 0.0f : __bfloat162float(__float2bfloat16_rn(w[off.V3 + u0 + k]));
        }
        for (int k = tid; k < 64; k += BT) b3[k] = (actor && k < O) ? w[off.b3 + k] : 0.0f;
        if (tid == 0) c3[0] = actor ? 0.0f : w[off.c3];
    };
    const size_t stride = a.agents ? (actor ? a.actor_stride : a.critic_stride) : 0;
    pack_weights(a.weights);
    int packed = 0;                                  // agent whose weights are packed
    for (int k = tid; k < BM * KX * 2 / 16; k += BT) st_shared_v4(smem + L.x + k * 16, 0u, 0u, 0u, 0u);
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, TMEM_COLS);
    sync_for_mma();
    cluster_sync();                                  // both CTAs run before any remote store
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t sx = smem_u32(smem + L.x), sh = smem_u32(smem + L.h);
    const uint32_t sw1 = smem_u32(smem + L.w1), sw2 = smem_u32(smem + L.w2), sw3 = smem_u32(smem + L.w3);
    // rank 0 of an actor cluster, once the head product is read: rank 1's partial
    // logits [BM][64] in the second half of the hidden operand, the sampler's
    // scratch in the first
    float* recv = (float*)(smem + L.h + BM * WD_HALF * 2);
    const int n_env = a.rows / a.per_env;
    const int tpa = (n_env + BM - 1) / BM;
    const int n_tiles = a.agents ? a.agents * tpa : (a.rows + BM - 1) / BM;
    const int t_lo = a.agents ? (int)((long long)n_tiles * role_pair / role_pairs) : role_pair;
    const int t_hi = a.agents ? (int)((long long)n_tiles * (role_pair + 1) / role_pairs) : n_tiles;
    const int t_step = a.agents ? 1 : role_pairs;
    uint32_t phase = 0;
    bool ok = true;
    for (int tile = t_lo; tile < t_hi; tile += t_step) {
        const int agent = a.agents ? tile / tpa : 0;
        const int e0 = a.agents ? (tile % tpa) * BM : 0;
        const int row0 = a.agents ? 0 : tile * BM;
        const int nrows = a.agents ? min(BM, n_env - e0) : min(BM, a.rows - row0);
        auto row_of = [&](int r) { return a.agents ? (e0 + r) * a.per_env + agent : row0 + r; };
        if (stride && agent != packed) {
            __syncthreads();                         // the previous tile's products are complete (waited)
            pack_weights(a.weights + (size_t)agent * stride);
            packed = agent;
        }
        // A failed wait skips the rest of the work, never a cluster barrier:
        // both CTAs pass the same barriers whatever happens.
        if (ok) {
            // observations -> BF16 operand [BM][KX]: a row per warp instruction (lane k:
            // column c0 + k of rows [16 warp, 16 warp + 16)), all of a warp's loads
            // issued before its stores; rows past the tile's end are zero
            for (int c0 = 0; c0 < I; c0 += 32) {
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int r = warp * 16 + q, k = c0 + lane;
                    v[q] = (r < nrows && k < I) ? __ldg(a.x + (size_t)row_of(r) * I + k) : 0.0f;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float nx = __shfl_down_sync(0xFFFFFFFFu, v[q], 1);
                    if ((lane & 1) == 0 && c0 + lane < KX)
                        st_shared_b32(smem + L.x + sw128_offset(warp * 16 + q, c0 + lane, BM), pack2(v[q], nx));
                }
            }
            sync_for_mma();
            if (tid == 0) {                          // layer 1, all 256 units: D[:, 0:256] = X W1
                mma_chain(tmem, sx, BM, sw1, WD_H, KX, idesc_bf16(BM, WD_H));
                mma_commit(&bar);
            }
            ok = wait_mma(&bar, phase);
        }
        if (ok) {
            for (int c = 0; c < 4; ++c) {            // this warpgroup's 128 units
                const int col = half * WD_HALF + c * 32;
                epilogue32(lane_base + col, b1 + col, smem + L.h, row, col);
            }
            sync_for_mma();
            if (tid == 0) {                          // layer 2, this rank's units: D[:, 0:128] = H1 W2[:, u0:u0+128]
                mma_chain(tmem, sh, BM, sw2, WD_HALF, WD_H, idesc_bf16(BM, WD_HALF));
                mma_commit(&bar);
            }
            ok = wait_mma(&bar, phase);
        }
        if (ok) {
            if (actor) {
                // H2 (this rank's units) into the first half of the hidden operand (H1 is read)
                for (int c = 0; c < 2; ++c) {
                    const int col = half * 64 + c * 32;
                    epilogue32(lane_base + col, b2 + col, smem + L.h, row, col);
                }
                sync_for_mma();
                if (tid == 0) {                      // partial logits over this rank's units
                    mma_chain(tmem + 256, sh, BM, sw3, 64, WD_HALF, idesc_bf16(BM, N3));
                    mma_commit(&bar);
                }
                ok = wait_mma(&bar, phase);
            } else {
                float vp = 0.0f;
                for (int c = 0; c < 2; ++c) {
                    const int col = half * 64 + c * 32;
                    vp += dot32(lane_base + col, b2 + col, v3r + col);
                }
                vpart[half][row] = vp;
                __syncthreads();
            }
        }
        cluster_sync();                              // H1 is dead in both; rank 0 is done with the last partials
        if (ok && rank == 1) {
            if (actor) {
                if (half * 32 < N3) {                // warp-uniform
                    float v[32];
                    tmem_ld32(lane_base + 256 + half * 32, v);
                    const uint32_t dst = cluster_addr(recv + row * WD_RECV + half * 32, 0);
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        if (half * 32 + j < O) st_cluster_v4(dst + 4 * j, v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
            } else if (half == 0) {
                st_cluster_f32(&vrecv[row], 0, vpart[0][row] + vpart[1][row]);
            }
        }
        cluster_sync();                              // rank 1's partials are in rank 0
        if (ok && rank == 0) {
            if (actor) {
                const bool live = row < nrows;
                // the logits: this rank's partial + rank 1's + the bias, back into the
                // head's TMEM columns, from where the sampler reads them
                if (half * 32 < N3) {
                    float v[32];
                    tmem_ld32(lane_base + 256 + half * 32, v);
                    const float4* rv = reinterpret_cast<const float4*>(recv + row * WD_RECV + half * 32);
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const float4 r4 = rv[j / 4];
                        const float4 b4 = *reinterpret_cast<const float4*>(b3 + half * 32 + j);
                        v[j] = (v[j] + r4.x) + b4.x; v[j + 1] = (v[j + 1] + r4.y) + b4.y;
                        v[j + 2] = (v[j + 2] + r4.z) + b4.z; v[j + 3] = (v[j + 3] + r4.w) + b4.w;
                    }
                    tmem_st32(lane_base + 256 + half * 32, v);
                    if (live && a.logits)
                        for (int j = 0; j < 32; ++j)
                            if (half * 32 + j < O) a.logits[(size_t)row_of(row) * O + half * 32 + j] = v[j];
                }
                tc_fence_before();
                __syncthreads();
                tc_fence_after();
                if (half == 0 && a.act) {
                    // mask words and uniforms of the row, as the pipelined kernel takes them
                    const int grow = live ? row_of(row) : 0;
                    uint32_t mw[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
                    float us[EJ_MAX_NB] = {0.0f, 0.0f, 0.0f, 0.0f};
                    if (live) {
                        if (a.W) {
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (k < a.W) mw[k] = a.mask[(size_t)grow * a.W + k];
                        }
                        if (a.u) {
#pragma unroll
                            for (int h = 0; h < EJ_MAX_NB; ++h)
                                if (h < a.n_heads) us[h] = a.u[(size_t)grow * a.n_heads + h];
                        } else {
                            const int e = a.env0 + grow / a.per_env, i = grow % a.per_env;
                            const uint4 x = philox4x32_10(make_uint4(a.stream_id == 0 ? (uint32_t)i : 0u, (uint32_t)e,
                                                                     a.gstep[e], (uint32_t)a.stream_id),
                                                          a.key[0], a.key[1]);
                            if (a.stream_id == 0) us[0] = u01(x.w);
                            else { us[0] = u01(x.x); us[1] = u01(x.y); us[2] = u01(x.z); us[3] = u01(x.w); }
                        }
                    }
                    // scratch: this thread's column of a [64][128] float array in the
                    // first half of the hidden operand (H2 is read); bias: zeros (v3r)
                    float* scr = reinterpret_cast<float*>(smem + L.h) + row;
                    float logp = 0.0f, ent = 0.0f;
                    bool none = false;
                    for (int h = 0; h < a.n_heads; ++h) {
                        const float uh = h == 0 ? us[0] : h == 1 ? us[1] : h == 2 ? us[2] : us[3];
                        int act = sample_head_tmem(lane_base + 256, v3r, h * a.head, a.head, mw, uh, scr, logp, ent);
                        if (act < 0) { act = 0; none = true; }
                        if (live) a.act[(size_t)grow * a.n_heads + h] = act;
                    }
                    if (none) { logp = 0.0f; ent = 0.0f; }
                    if (live) {
                        a.logp[grow] = logp;
                        if (a.entropy) a.entropy[grow] = ent;
                    }
                }
            } else if (half == 0 && row < nrows) {
                a.value[row_of(row)] = ((vpart[0][row] + vpart[1][row]) + vrecv[row]) + c3[0];
            }
        }
    }
    if (!ok) mbar_wait(&bar, phase, 200000000LL);   // one more bounded chance before freeing TMEM
    cluster_sync();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem_slot, TMEM_COLS);
}

ej_status launch_policy_bf16_wide(const PolicyArgs& a, cudaStream_t stream) {
    if (a.in_dim > KX) return fail(EJ_ERR_UNSUPPORTED, "bf16 policy: input width must be <= %d", KX);
    if (a.O > WD_MAX_O) return fail(EJ_ERR_UNSUPPORTED, "bf16 policy: at most %d logits at hidden %d", WD_MAX_O, WD_H);
    if (a.n_heads < 1 || a.n_heads > EJ_MAX_NB) return fail(EJ_ERR_UNSUPPORTED, "bf16 policy: 1 to %d heads", EJ_MAX_NB);
    const size_t smem = wd_layout().total + 1024;
    static SmemOptIn opt_in;
    ej_status st = opt_in.ensure((const void*)policy_bf16_wide_kernel, smem);
    if (st != EJ_OK) return st;
    // clusters of two CTAs, one CTA per SM; the actor's tile costs about 17.7 k
    // SM cycles against the critic's 10.7 k (clock64 stamps per phase, GB300,
    // 24 logits): the actor clusters' share balances the two roles
    int pairs = device_sms() / 2 >= 2 ? device_sms() / 2 : 2;
    {
        // as many clusters as can be resident at once (a GPC may leave an SM unpaired)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * pairs);
        cfg.blockDim = dim3(BT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        int resident = 0;
        if (cudaOccupancyMaxActiveClusters(&resident, (const void*)policy_bf16_wide_kernel, &cfg) == cudaSuccess &&
            resident >= 2 && resident < pairs)
            pairs = resident;
        cudaGetLastError();
    }
    int n_act = (int)(pairs * (17.7 / (17.7 + 10.7)) + 0.5);
    n_act = n_act < 1 ? 1 : (n_act > pairs - 1 ? pairs - 1 : n_act);
    policy_bf16_wide_kernel<<<2 * pairs, BT, smem, stream>>>(a, n_act);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "bf16 policy (hidden 256) launch: %s", cudaGetErrorString(err));
    return EJ_OK;
}

ej_status launch_policy_bf16(const PolicyArgs& a, cudaStream_t stream) {
    if (a.H == WD_H) return launch_policy_bf16_wide(a, stream);
    if (a.H != 64 && a.H != 128) return fail(EJ_ERR_UNSUPPORTED, "bf16 policy: hidden must be 64, 128 or 256");
    if (a.in_dim > KX) return fail(EJ_ERR_UNSUPPORTED, "bf16 policy: input width must be <= %d", KX);
    if (a.O > 128) return fail(EJ_ERR_UNSUPPORTED, "bf16 policy: at most 128 logits");
    if ((a.O | 1) > a.H) return fail(EJ_ERR_UNSUPPORTED, "bf16 policy: logits do not fit the staging area");
    const size_t smem = policy_bf16_smem(a.H, a.O);
    if (smem > 227 * 1024) return fail(EJ_ERR_UNSUPPORTED, "bf16 policy: %zu bytes of shared memory", smem);
    static SmemOptIn opt_in;
    ej_status st_opt = opt_in.ensure((const void*)policy_bf16_kernel, smem);
    if (st_opt != EJ_OK) return st_opt;
    const int n_tiles = a.agents ? a.agents * ((a.rows / a.per_env + BM - 1) / BM) : (a.rows + BM - 1) / BM;
    int grid = n_tiles < device_sms() ? n_tiles : device_sms();
    if (grid < 1) grid = 1;
    if (a.agents) {
        // per-agent networks: the general kernel, agent-major tiles, weights packed per agent
        policy_bf16_kernel<<<grid, BT, smem, stream>>>(a);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "bf16 policy launch: %s", cudaGetErrorString(err));
        return EJ_OK;
    }
    if (a.H == 128) {
        bool handled = false;
        ej_status st = launch_policy_bf16_multi(&a, 1, stream, &handled);
        if (st != EJ_OK || handled) return st;
    }
    const bool fast = a.O <= 64 && a.in_dim <= 32 && a.W <= 2 && a.n_heads <= EJ_MAX_NB && ((uintptr_t)a.x & 15) == 0;
    if (fast) {
        static SmemOptIn opt_fast[2];
        const int kt = a.O <= 32 ? 0 : 1;
        ej_status st_fast = opt_fast[kt].ensure(
            kt == 0 ? (const void*)policy_bf16_fast_kernel<32> : (const void*)policy_bf16_fast_kernel<64>, smem);
        if (st_fast != EJ_OK) return st_fast;
        if (kt == 0) policy_bf16_fast_kernel<32><<<grid, BT, smem, stream>>>(a);
        else policy_bf16_fast_kernel<64><<<grid, BT, smem, stream>>>(a);
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "bf16 policy launch: %s", cudaGetErrorString(err));
        return EJ_OK;
    }
    policy_bf16_kernel<<<grid, BT, smem, stream>>>(a);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "bf16 policy launch: %s", cudaGetErrorString(err));
    return EJ_OK;
}

}  // namespace ej

extern "C" ej_status ej_device_status(int32_t* fault, int32_t clear) {
    int v = 0;
    cudaError_t err = cudaMemcpyFromSymbol(&v, ej::g_ej_fault, sizeof(int));
    if (err != cudaSuccess) return ej::fail(EJ_ERR_CUDA, "ej_device_status: %s", cudaGetErrorString(err));
    v |= ej::ppo_bf16_fault(clear);
    if (fault) *fault = v;
    if (clear) {
        const int z = 0;
        err = cudaMemcpyToSymbol(ej::g_ej_fault, &z, sizeof(int));
        if (err != cudaSuccess) return ej::fail(EJ_ERR_CUDA, "ej_device_status: %s", cudaGetErrorString(err));
    }
    return EJ_OK;
}
