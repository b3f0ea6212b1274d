// Policy forward / sampling: shared declarations of the float32 and bf16 paths.
#pragma once

#include <cfloat>

#include "ej_internal.cuh"

namespace ej {

// Offsets of the parameter vector of one network (actor then critic):
// W1 [in][H], b1 [H], W2 [H][H], b2 [H], W3 [H][O], b3 [O],
// V1 [in][H], c1 [H], V2 [H][H], c2 [H], V3 [H], c3 [1]; every tensor starts
// at a multiple of 4 floats (16 bytes), the gaps are padding.
struct NetOffsets {
    size_t W1, b1, W2, b2, W3, b3, V1, c1, V2, c2, V3, c3, total;
};

__host__ __device__ inline size_t pad4(size_t x) { return (x + 3) & ~size_t(3); }

__host__ __device__ inline NetOffsets net_offsets(int in, int H, int O) {
    NetOffsets o;
    size_t p = 0;
    o.W1 = p; p = pad4(p + (size_t)in * H);
    o.b1 = p; p = pad4(p + H);
    o.W2 = p; p = pad4(p + (size_t)H * H);
    o.b2 = p; p = pad4(p + H);
    o.W3 = p; p = pad4(p + (size_t)H * O);
    o.b3 = p; p = pad4(p + O);
    o.V1 = p; p = pad4(p + (size_t)in * H);
    o.c1 = p; p = pad4(p + H);
    o.V2 = p; p = pad4(p + (size_t)H * H);
    o.c2 = p; p = pad4(p + H);
    o.V3 = p; p = pad4(p + H);
    o.c3 = p; p = pad4(p + 1);
    o.total = p;
    return o;
}

struct PolicyArgs {
    int rows;            // rows of x (E*A for the population, E for the government)
    int per_env;         // rows per environment (A or 1)
    int in_dim, in_pad;  // observation width and its padding to a multiple of 4
    int H, O;            // hidden units, logits per row (n_heads * head)
    int n_heads, head;   // population: 1 head of nA (masked); government: nb heads of tax_levels
    int W;               // mask words per row (0: every action allowed)
    int stream_id;       // Philox stream of the sampling uniforms (0 population, 1 government)
    int env0;            // global index of the first environment of x's rows (Philox counters)
    const float* weights;
    const float* x;
    const uint32_t* mask;
    const float* u;               // [rows][n_heads] or NULL: Philox at the state's global step
    const uint32_t* gstep;        // state: global step per environment
    const uint32_t* key;          // state: Philox key
    int32_t* act;                 // [rows][n_heads] or NULL (no sampling)
    float* logp;                  // [rows] sum over heads
    float* value;                 // [rows]
    float* entropy;               // [rows] sum over heads (may be NULL)
    float* logits;                // [rows][O] (may be NULL)
    // Per-agent networks of the population (Section 5): agents > 0 gives each
    // of the per_env agents its own actor (weights + i * actor_stride) and
    // critic (weights + i * critic_stride; stride 0: one shared critic), and
    // the kernel takes agent-major tiles (one agent, TILE environments).
    int agents;
    size_t actor_stride, critic_stride;
};

// Row segments of one policy launch: several buffers (e.g. several
// environment classes that share a network) processed by one grid.  Each
// segment's rows are padded to whole 128-row tiles; tile0 = its first tile
// within its network's tiles.
constexpr int EJ_MAX_SEG = 32;
constexpr int EJ_MAX_NET = 4;
struct PolicySeg {
    const float* x;
    const uint32_t* mask;
    const float* u;
    const uint32_t* gstep;
    const uint32_t* key;
    int32_t* act;
    float* logp;
    float* value;
    float* entropy;
    float* logits;
    int rows, per_env, tile0;
    int env0;         // global index of the segment's first environment (its Philox counters)
};
// A network of a launch: its weights and shape, its segments
// [seg_lo, seg_hi) and its CTAs (actors [cta0, cta0 + n_act), critics after).
struct PolicyNet {
    const float* weights;
    int in_dim, O, n_heads, head, W, stream_id;
    int seg_lo, seg_hi, n_tiles;
    int cta0, n_act, n_cri;
};
struct PolicyLaunch {
    int H, n3_max, n_net, n_seg;
    PolicyNet net[EJ_MAX_NET];
    PolicySeg seg[EJ_MAX_SEG];
};

// One launch of the pipelined BF16 kernel over segs[0..n) (each a PolicyArgs
// of its own rows; segments with the same weights and shape form one
// network, at most EJ_MAX_NET networks and EJ_MAX_SEG segments).  *handled =
// false (nothing launched) when a shape is outside the kernel's range
// (hidden 128, <= 96 logits, <= 32 inputs, <= 4 mask words) or an
// observation buffer is not 4-byte aligned.
ej_status launch_policy_bf16_multi(const PolicyArgs* segs, int n, cudaStream_t stream, bool* handled);

// exp on float32 by Cody-Waite reduction (Cody and Waite, "Software Manual for
// the Elementary Functions", 1980) and the degree-7 Taylor polynomial of e^r
// on |r| <= ln2/2, Horner's rule, each operation rounded once; 0 below -80.
__device__ __forceinline__ float exp32(float x) {
    if (x < -80.0f) return 0.0f;
    const float n = rintf(__fmul_rn(x, 0x1.715476p+0f));
    float r = __fsub_rn(x, __fmul_rn(n, 0x1.62e4p-1f));
    r = __fsub_rn(r, __fmul_rn(n, 0x1.7f7d1cp-20f));
    float p = 0x1.a01a02p-13f;
    p = __fadd_rn(__fmul_rn(p, r), 0x1.6c16c2p-10f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.111112p-7f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-5f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-3f);
    p = __fadd_rn(__fmul_rn(p, r), 0.5f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    const int ni = (int)n;
    return __fmul_rn(p, __int_as_float((ni + 127) << 23));
}

// Inverse-CDF draw of one head from its logits l[0..K) under `valid` bits.
// Returns the action (-1 if nothing is allowed) and adds the head's log
// probability and entropy.  w[0..K) is scratch for the exp weights (each is
// computed once and reused for the draw); NULL: they are recomputed.
__device__ __forceinline__ int sample_head(const float* l, int K, const uint32_t* valid_words,
                                           int bit0, float u, float& logp, float& ent, float* w) {
    float m = -FLT_MAX;
    bool any = false;
    for (int j = 0; j < K; ++j) {
        const bool ok = !valid_words || ((valid_words[(bit0 + j) >> 5] >> ((bit0 + j) & 31)) & 1u);
        if (ok) { any = true; m = fmaxf(m, l[j]); }
    }
    if (!any) return -1;
    float S = 0.0f, dot = 0.0f;
    for (int j = 0; j < K; ++j) {
        const bool ok = !valid_words || ((valid_words[(bit0 + j) >> 5] >> ((bit0 + j) & 31)) & 1u);
        float wj = 0.0f;
        if (ok) {
            const float d = __fsub_rn(l[j], m);
            wj = exp32(d);
            S = __fadd_rn(S, wj);
            dot = fmaf(wj, d, dot);
        }
        if (w) w[j] = ok ? wj : -1.0f;          // -1 marks a forbidden action
    }
    const float thr = __fmul_rn(u, S);
    float c = 0.0f;
    int act = -1, last = -1;
    for (int j = 0; j < K; ++j) {
        float wj;
        if (w) {
            wj = w[j];
        } else {                                 // no scratch: the same weights, recomputed
            const bool ok = !valid_words || ((valid_words[(bit0 + j) >> 5] >> ((bit0 + j) & 31)) & 1u);
            wj = ok ? exp32(__fsub_rn(l[j], m)) : -1.0f;
        }
        if (wj >= 0.0f) {
            last = j;
            c = __fadd_rn(c, wj);
            if (act < 0 && c > thr) act = j;
        }
    }
    if (act < 0) act = last;
    const float logS = logf(S);
    logp += (l[act] - m) - logS;
    ent += logS - dot / S;
    return act;
}

// Outputs of one row's actor: the logits (when asked for) and, when sampling,
// the actions, log probability and entropy of its heads.
__device__ __forceinline__ void sample_row_act(const PolicyArgs& a, int row, const float* l, float* w) {
    if (a.logits)
        for (int j = 0; j < a.O; ++j) a.logits[(size_t)row * a.O + j] = l[j];
    if (!a.act) return;
    const int e = a.env0 + row / a.per_env, i = row % a.per_env;
    float us[EJ_MAX_NB];
    if (a.u) {
        for (int h = 0; h < a.n_heads; ++h) us[h] = a.u[(size_t)row * a.n_heads + h];
    } else {
        const uint32_t g = a.gstep[e];
        const uint4 x = philox4x32_10(make_uint4(a.stream_id == 0 ? (uint32_t)i : 0u, (uint32_t)e, g,
                                                 (uint32_t)a.stream_id), a.key[0], a.key[1]);
        if (a.stream_id == 0) us[0] = u01(x.w);
        else { us[0] = u01(x.x); us[1] = u01(x.y); us[2] = u01(x.z); us[3] = u01(x.w); }
    }
    float logp = 0.0f, ent = 0.0f;
    const uint32_t* mw = a.W ? a.mask + (size_t)row * a.W : nullptr;
    bool none = false;
    for (int h = 0; h < a.n_heads; ++h) {
        int act = sample_head(l + h * a.head, a.head, mw, h * a.head, us[h < EJ_MAX_NB ? h : 0], logp, ent, w);
        if (act < 0) { act = 0; none = true; }
        a.act[(size_t)row * a.n_heads + h] = act;
    }
    if (none) { logp = 0.0f; ent = 0.0f; }
    a.logp[row] = logp;
    if (a.entropy) a.entropy[row] = ent;
}

__device__ __forceinline__ void sample_row(const PolicyArgs& a, int row, const float* l, float value, float* w) {
    a.value[row] = value;
    sample_row_act(a, row, l, w);
}

// Row tiles of the SIMT (float32) network kernels.
constexpr int TILE = 64;       // rows per tile
constexpr int NTH = 256;       // threads per CTA

// Visits (r, c) for r < ROWS, c < ncols (ncols <= NTH): thread t takes
// column t % ncols of rows t / ncols, t / ncols + NTH / ncols, ... (one
// division per call rather than per element).  Every caller passes at most
// NTH columns: padded inputs (at most 124: 16 resources), hidden widths (at
// most 256) or a quarter of them, logits (at most 128 in the PPO kernels).
template <int ROWS, class F>
__device__ __forceinline__ void tile_for(int ncols, F&& f) {
    const int per = NTH / ncols, r0 = (int)threadIdx.x / ncols;
    if (r0 >= per) return;
    const int c = (int)threadIdx.x - r0 * ncols;
    for (int r = r0; r < ROWS; r += per) f(r, c);
}

// out[r][c] = act(b[c] + sum_k in[r][k] W[k][c]) for a ROWS x N block, N a
// multiple of 32 (the hidden width); b may be NULL (no bias).  Thread tile: RT
// rows x 4 columns, the rows strided by ROWS / RT.  in: 16-byte aligned, ldi a
// multiple of 4.  A warp covers 8 column groups x 4 row groups: per k it reads
// 128 contiguous weight bytes (one L1 wavefront, where 32 column groups would
// take four) and 4 consecutive input rows, on distinct banks for row pitches
// of 4 to 28 floats mod 32.  Each output still sums its k in order.
template <int ROWS = TILE, int RT = 8>
__device__ inline void dense_tile(const float* in, int ldi, int K, const float* __restrict__ W,
                           const float* __restrict__ b, int N, float* out, int ldo, bool relu) {
    constexpr int RG = ROWS / RT;              // row groups
    static_assert(RG % 4 == 0, "a warp covers 4 row groups");
    const int cb = N >> 5;                     // warp tiles across the columns
    for (int base = threadIdx.x; base < (N >> 2) * RG; base += NTH) {
        const int lane = base & 31, blk = base >> 5;
        const int bc = blk % cb;
        const int c0 = (bc * 8 + (lane & 7)) * 4;
        const int rg = (blk - bc) / cb * 4 + (lane >> 3);
        float acc[RT][4];
        const float4 bb = b ? *reinterpret_cast<const float4*>(b + c0) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < RT; ++r) { acc[r][0] = bb.x; acc[r][1] = bb.y; acc[r][2] = bb.z; acc[r][3] = bb.w; }
        const float* x0 = in + rg * ldi;
        // four k per step: 16-byte loads of the inputs (ldi is a multiple of 4),
        // four weight rows in flight; each accumulator still takes its k in order
        int k = 0;
#pragma unroll 2
        for (; k + 4 <= K; k += 4) {
            float4 w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = __ldg(reinterpret_cast<const float4*>(W + (size_t)(k + q) * N + c0));
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const float4 x4 = *reinterpret_cast<const float4*>(x0 + r * RG * ldi + k);
                const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[r][0] = fmaf(xs[q], w[q].x, acc[r][0]);
                    acc[r][1] = fmaf(xs[q], w[q].y, acc[r][1]);
                    acc[r][2] = fmaf(xs[q], w[q].z, acc[r][2]);
                    acc[r][3] = fmaf(xs[q], w[q].w, acc[r][3]);
                }
            }
        }
        for (; k < K; ++k) {
            const float4 w = __ldg(reinterpret_cast<const float4*>(W + (size_t)k * N + c0));
#pragma unroll
            for (int r = 0; r < RT; ++r) {
                const float x = x0[r * RG * ldi + k];
                acc[r][0] = fmaf(x, w.x, acc[r][0]);
                acc[r][1] = fmaf(x, w.y, acc[r][1]);
                acc[r][2] = fmaf(x, w.z, acc[r][2]);
                acc[r][3] = fmaf(x, w.w, acc[r][3]);
            }
        }
#pragma unroll
        for (int r = 0; r < RT; ++r) {
            float4 v = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            if (relu) { v.x = fmaxf(v.x, 0.0f); v.y = fmaxf(v.y, 0.0f); v.z = fmaxf(v.z, 0.0f); v.w = fmaxf(v.w, 0.0f); }
            *reinterpret_cast<float4*>(out + (rg + r * RG) * ldo + c0) = v;
        }
    }
}

// Output head of width O (any): one thread per (row, column), IPT of them
// in flight per thread (independent chains; each sums its k in order).
template <int ROWS = TILE, int IPT = 1>
__device__ inline void head_tile(const float* in, int ldi, int K, const float* __restrict__ W,
                          const float* __restrict__ b, int O, float* out, int ldo) {
    const int n = ROWS * O;
    if constexpr (IPT == 1) {
        for (int idx = threadIdx.x; idx < n; idx += NTH) {
            const int r = idx / O, c = idx % O;
            float acc = b[c];
            const float* x = in + r * ldi;
#pragma unroll 8
            for (int k = 0; k < K; ++k) acc = fmaf(x[k], __ldg(W + (size_t)k * O + c), acc);
            out[r * ldo + c] = acc;
        }
        return;
    }
    for (int base = threadIdx.x; base < n; base += NTH * IPT) {
        float acc[IPT];
        const float* x[IPT];
        int c[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int idx = min(base + j * NTH, n - 1);     // past the end: recompute the last, not stored
            c[j] = idx % O;
            x[j] = in + (idx / O) * ldi;
            acc[j] = b[c[j]];
        }
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
            const float* wk = W + (size_t)k * O;
#pragma unroll
            for (int j = 0; j < IPT; ++j) acc[j] = fmaf(x[j][k], __ldg(wk + c[j]), acc[j]);
        }
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int idx = base + j * NTH;
            if (idx < n) out[(idx / O) * ldo + idx % O] = acc[j];
        }
    }
}

// Critic output: one warp per row, lanes split the hidden units.
template <int ROWS = TILE>
__device__ inline void value_tile(const float* in, int ldi, int K, const float* __restrict__ v,
                           float c, float* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < ROWS; r += NTH / 32) {
        float acc = 0.0f;
        for (int k = lane; k < K; k += 32) acc = fmaf(in[r * ldi + k], __ldg(v + k), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) out[r] = acc + c;
    }
}

size_t policy_fp32_smem(int in_pad, int H, int O);
ej_status launch_policy_fp32(const PolicyArgs& a, cudaStream_t stream);
size_t policy_bf16_smem(int H, int O);
ej_status launch_policy_bf16(const PolicyArgs& a, cudaStream_t stream);
// One launch over several row segments sharing the network of `a` (a's own
// row pointers are ignored); false in *handled when the shape has no
// segmented kernel (the caller then launches per segment).

}  // namespace ej
