// PPO minibatch gradient on the 5th-generation tensor cores: BF16 operands,
// FP32 accumulation in tensor memory (tcgen05.mma kind::f16, M = 128).
//
// The loss of Section 4 separates: the clipped surrogate and the entropy
// bonus depend only on the actor, the clipped value loss only on the critic
// (the advantages come from GAE on the rollout's values).  So the grid is
// split: CTAs [0, n_actor) run the actor, the others the critic, each
// persistent over 128-row tiles of the minibatch (one CTA per SM).
//
// Per tile, everything stays on chip: forward layers (MMA, then an epilogue
// that adds the bias, applies ReLU and writes the BF16 activation back to
// shared memory as the next operand; the backward masks read it there), the
// loss gradient per row, the backward-data products, and the weight-gradient
// products.  The weight gradients of all tiles accumulate in tensor memory
// (they are sums over rows, i.e. MMAs with K = rows): dW = A^T dZ reads the
// stored activation tiles as MN-major (transposed) operands, so no transposed
// copy is ever written.  Bias gradients come with the weight gradients: the
// second layer's as the transposed product dW2^T | db2 = dZ2^T [H1 | 1] (an
// all-ones panel follows H1 in shared memory), the first layer's from the
// inputs' ones column, the head's against an all-ones operand; the value
// head's bias gradient (a plain sum of dv) on the CUDA cores.
// Each backward-data product (dZ2, dZ1) is committed on its own and the
// weight-gradient products issued behind it, so an epilogue waits only for
// the product it reads; the weight-gradient products finish under the next
// epilogue (a commit covers every earlier product, which orders them before
// the buffers they read are overwritten).  The critic's value head (one
// output column) is a dot product in the second layer's epilogue.
// At the end each CTA writes its accumulators once; a reduction kernel sums
// the CTAs into the gradient vector.
//
// Operand layouts: every tile buffer is [rows][cols] BF16 in the 128-byte
// swizzled K-major layout of sw128_offset (panels of 64 columns).  Read with
// K along the columns it is a K-major operand; read with K along the rows
// (weight gradients, and weights multiplied transposed in the backward pass)
// it is an MN-major operand whose leading byte offset is the panel stride and
// whose stride byte offset is one 8-row atom (1024 bytes).
#include <cfloat>
#include <cmath>
#include <cstring>

#include "ej_internal.cuh"
#include "ej_policy.cuh"
#include "ej_ppo.cuh"

namespace ej {
namespace {
__device__ int g_ej_fault = 0;   // set when a bounded wait of this file's kernel gives up
}
}  // namespace ej

#include "ej_tc.cuh"

namespace ej {

namespace {

constexpr int BM = 128;        // rows per tile = TMEM lanes
constexpr int BT = 256;        // threads: two warpgroups share the 128 lanes (64 columns each)
constexpr int HID = 128;       // hidden width of this path
constexpr int KX = 64;         // input operand width: inputs, then a ones column (bias gradients)
constexpr int KO = 64;         // logit operand width
constexpr uint32_t TMEM_COLS = 512;
constexpr int PC = 352;        // accumulator columns written per TMEM lane
// Cost of a tile in thousands of SM cycles, measured with clock64 stamps per
// phase on GB300 (population minibatch of E = 2048 x A = 100 x 128 steps):
// about 11.9 for the critic (inputs, two forward products and epilogues with
// the value head, value loss, backward products and masks); the actor adds
// its head product and the loss: 4.5 with at most 32 logits (registers), and
// for wider heads about 1.9 per group of 8 logit columns they span (three
// heads of 21: 18.4).
constexpr double PPO_TILE = 11.9, PPO_LOSS_REG = 4.5, PPO_LOSS_GROUP = 1.9;

// TMEM columns.  Actor: dW1^T [h][in] 0..63, dW2^T [h_out][h_in] 64..191 and
// db2 (192, from the same product: dZ2^T [H1 | 1]), dW3 [h][o] 208..271, db3
// [o] 272..335 (every lane).  Critic: dV1^T 0..63, dV2^T 64..191 and dc2 (192),
// dV3 (208); dc3 is summed on the CUDA cores and stored at column 224 of the
// CTA's partial row 0.  Both: per-tile products in 384..511.
constexpr uint32_t C_W1T = 0, C_W2 = 64, C_B2 = 192, C_W3 = 208, C_B3 = 272;
constexpr uint32_t C_C2 = 192, C_V3 = 208, C_C3 = 224;
constexpr uint32_t C_SLOT = 384;

// Shared memory (bytes from the 1024-aligned base).
struct PpoSmem {
    uint32_t w1, w2, w3, x, h1, h2, dl, dz2, ones, dv, bias, total;
};

// Actor and critic use the same regions under different names:
//   w1: W1 / V1 [128][KX]        w2: W2 / V2 [128][128]      w3: W3 [KO][128] (actor)
//   x:  inputs [128][KX]         h1: H1 / G1 [128][128]      h2: H2 / G2, later dZ1 / dY1
//   dl: dL [128][KO] (actor)     dz2: dZ2 / dY2 [128][128]   dv: dv [16][128] (critic)
//   ones: all-ones [128][64] (follows h1)     bias: floats
__host__ __device__ inline PpoSmem ppo_smem() {
    PpoSmem L;
    uint32_t b = 0;
    L.w1 = b;   b += HID * KX * 2;
    L.w2 = b;   b += HID * HID * 2;
    L.w3 = b;   b += KO * HID * 2;
    L.x = b;    b += BM * KX * 2;
    L.h1 = b;   b += BM * HID * 2;
    L.ones = b; b += BM * 64 * 2;      // right after H1: [H1 | 1] is one MN-major operand of 192 columns
    L.h2 = b;   b += BM * HID * 2;
    L.dl = b;   b += BM * KO * 2;
    L.dz2 = b;  b += BM * HID * 2;
    L.dv = b;   b += 16 * BM * 2;
    L.bias = b; b += (3 * HID + KO + 2 * BM + HID + 2 * BM) * 4;
    L.total = b;
    return L;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// A read-only global load issued where it is written (volatile: the compiler
// does not move it next to its use), so a prefetch stays a prefetch.
__device__ __forceinline__ float ld_nc_issue(const float* p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_nc_issue(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int32_t ld_nc_issue(const int32_t* p) {
    int32_t v;
    asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Hint: bring the line holding p into L2 (no result, nothing waits for it).
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void st_shared_u32(uint8_t* p, uint32_t a) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(smem_u32(p)), "r"(a) : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint8_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(p)), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Shared-memory descriptor of a 128-byte swizzled operand with explicit
// leading and stride byte offsets.
__device__ __forceinline__ uint64_t sw128_desc_ls(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Descriptor of a K-major operand (K along the columns of a buffer).
__device__ __forceinline__ uint64_t kdesc(uint32_t base) { return sw128_desc(base); }
// Descriptor of an MN-major operand: a buffer of ROWS rows read with K along the rows.
template <int ROWS>
__device__ __forceinline__ uint64_t mndesc(uint32_t base) { return sw128_desc_ls(base, (ROWS / 8) * 1024, 1024); }

constexpr uint32_t TA = 1u << 15, TB = 1u << 16;   // MN-major A / B in the instruction descriptor

// Walks of an operand over K steps of 16.  The start-address field of a
// shared-memory descriptor (bits 0-13: address / 16) does not carry out for
// addresses below 256 KB, so the descriptor of base + off is the base's plus
// off / 16: one add per step.
enum : int {
    K_MAJ = 0,     // K-major buffer of R rows: 64-column panels of R / 8 atoms, 32 bytes per step in a panel
    MN_MAJ = 1,    // MN-major: the next 16 rows, 2048 bytes on
    K_ONE = 2,     // K-major, the steps of one 64-column panel repeated (the all-ones operand)
};
template <int KIND, int R>
__device__ __forceinline__ uint32_t kstep(int kk) {
    return KIND == MN_MAJ ? (uint32_t)kk * 128u
                          : (KIND == K_ONE ? 0u : (uint32_t)(kk >> 2) * (uint32_t)(R * 8)) + (uint32_t)(kk & 3) * 2u;
}

// D (+)= A B over KS steps of K = 16, the operands' descriptors walked from a and b.
template <int KS, int AK, int AR, int BK, int BR>
__device__ __forceinline__ void chain(uint32_t d, uint32_t idesc, bool acc, uint64_t a, uint64_t b) {
#pragma unroll
    for (int kk = 0; kk < KS; ++kk)
        mma_bf16(d, a + kstep<AK, AR>(kk), b + kstep<BK, BR>(kk), idesc, (acc || kk > 0) ? 1u : 0u);
}

__device__ __forceinline__ void sync_for_mma() {
    fence_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

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

// Packs rows x K of a K-major operand from a float source get(n, k).
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

// 64 consecutive accumulator columns of this thread's TMEM lane (two loads, one wait).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
    uint32_t r[64];
#define EJ_LD32(OFF, B)                                                                                         \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "                                                    \
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"                                     \
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                    \
                 : "=r"(r[B + 0]), "=r"(r[B + 1]), "=r"(r[B + 2]), "=r"(r[B + 3]), "=r"(r[B + 4]),             \
                   "=r"(r[B + 5]), "=r"(r[B + 6]), "=r"(r[B + 7]), "=r"(r[B + 8]), "=r"(r[B + 9]),             \
                   "=r"(r[B + 10]), "=r"(r[B + 11]), "=r"(r[B + 12]), "=r"(r[B + 13]), "=r"(r[B + 14]),        \
                   "=r"(r[B + 15]), "=r"(r[B + 16]), "=r"(r[B + 17]), "=r"(r[B + 18]), "=r"(r[B + 19]),        \
                   "=r"(r[B + 20]), "=r"(r[B + 21]), "=r"(r[B + 22]), "=r"(r[B + 23]), "=r"(r[B + 24]),        \
                   "=r"(r[B + 25]), "=r"(r[B + 26]), "=r"(r[B + 27]), "=r"(r[B + 28]), "=r"(r[B + 29]),        \
                   "=r"(r[B + 30]), "=r"(r[B + 31])                                                            \
                 : "r"(OFF))
    EJ_LD32(taddr, 0);
    EJ_LD32(taddr + 32, 32);
#undef EJ_LD32
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 64; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }
__device__ __forceinline__ __nv_bfloat162 bits_bf2(uint32_t u) { return *reinterpret_cast<__nv_bfloat162*>(&u); }

// 64 accumulator columns [col, col+64) of this thread's row: add the bias,
// round to BF16 pairs, ReLU on the pairs (max with 0 commutes with the
// rounding), write to columns [col, col+64) of dst.
// With dot != nullptr it also returns the sum over these columns of the
// BF16 activation times dot[k] (the critic's value head: dot holds the
// BF16-rounded V3 entries, so each product is the one the tensor core forms).
__device__ __forceinline__ float relu_epilogue64(uint32_t taddr, const float* bias, uint8_t* dst, int row, int col,
                                                 const float* dot = nullptr) {
    float v[64];
    tmem_ld64(taddr, v);
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        // bias on float32 pairs (add.rn.f32x2: each element rounded once), then
        // ReLU and BF16 in one conversion (the values of round-then-ReLU)
        const float4 b0 = *reinterpret_cast<const float4*>(bias + q * 8);
        const float4 b1 = *reinterpret_cast<const float4*>(bias + q * 8 + 4);
        float* y = v + q * 8;
        uint32_t w[4];
        const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            unsigned long long x, c, z;
            asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(y[2 * j]), "f"(y[2 * j + 1]));
            asm("mov.b64 %0, {%1, %2};" : "=l"(c) : "f"(bb[2 * j]), "f"(bb[2 * j + 1]));
            asm("add.rn.f32x2 %0, %1, %2;" : "=l"(z) : "l"(x), "l"(c));
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(z));
            asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(w[j]) : "f"(hi), "f"(lo));
        }
        st_shared_v4(dst + sw128_offset(row, col + q * 8, BM), w[0], w[1], w[2], w[3]);
        if (dot) {
            const float4 d0 = *reinterpret_cast<const float4*>(dot + q * 8);
            const float4 d1 = *reinterpret_cast<const float4*>(dot + q * 8 + 4);
            const float dd[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc = fmaf(__uint_as_float(w[j] << 16), dd[2 * j], acc);
                acc = fmaf(__uint_as_float(w[j] & 0xFFFF0000u), dd[2 * j + 1], acc);
            }
        }
    }
    return acc;
}

// 64 accumulator columns times the ReLU derivative of the activation stored
// in act (BF16, same row and columns: [h > 0]) -> BF16 columns of dst.
__device__ __forceinline__ void mask_epilogue64(uint32_t taddr, const uint8_t* act, uint8_t* dst, int row, int col) {
    float v[64];
    tmem_ld64(taddr, v);
    const __nv_bfloat162 zero = __floats2bfloat162_rn(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint4 h = *reinterpret_cast<const uint4*>(act + sw128_offset(row, col + q * 8, BM));
        const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = q * 8 + 2 * j;
            w[j] = bf2_bits(__hmul2(__floats2bfloat162_rn(v[k], v[k + 1]), __hgt2(bits_bf2(hw[j]), zero)));
        }
        st_shared_v4(dst + sw128_offset(row, col + q * 8, BM), w[0], w[1], w[2], w[3]);
    }
}

struct BfPpoArgs {
    FbArgs f;
    float* partial;   // [grid][BM][PC] accumulators of each CTA
    int n_actor;      // CTAs [0, n_actor) run the actor, the rest the critic
};

// Up to four per-head values in registers (heads <= EJ_MAX_NB), indexed by a
// uniform head number without local memory.
struct Head4 {
    float v0 = 0.0f, v1 = 0.0f, v2 = 0.0f, v3 = 0.0f;
    __device__ __forceinline__ void set(int h, float x) {
        if (h == 0) v0 = x; else if (h == 1) v1 = x; else if (h == 2) v2 = x; else v3 = x;
    }
    __device__ __forceinline__ float get(int h) const { return h == 0 ? v0 : h == 1 ? v1 : h == 2 ? v2 : v3; }
};

struct ActorRow { float pg, ent, clip, kl; };

// Per-row inputs of the actor's loss, loaded at the start of a tile so that
// their latency overlaps the forward products.
struct RowIn {
    uint32_t w0, w1;           // action-mask words (all ones without a mask)
    int act0, act1, act2, act3;   // actions of heads 0..3
    float lpo, adv;            // log-probability at sampling time, raw advantage
    __device__ __forceinline__ int act(int h) const { return h == 0 ? act0 : h == 1 ? act1 : h == 2 ? act2 : act3; }
};

__device__ __forceinline__ RowIn load_row_in(const FbArgs& a, uint32_t row, bool two_words) {
    RowIn q;
    q.w0 = 0xFFFFFFFFu;
    q.w1 = 0xFFFFFFFFu;
    if (a.W) {
        const uint32_t* mw = a.mask + (size_t)row * a.W;
        q.w0 = ld_nc_issue(mw);
        q.w1 = 0u;
        if (two_words && a.W > 1) q.w1 = ld_nc_issue(mw + 1);
    }
    const int32_t* ac = a.act + (size_t)row * a.n_heads;
    q.act0 = ld_nc_issue(ac);
    q.act1 = q.act2 = q.act3 = 0;
    if (a.n_heads > 1) q.act1 = ld_nc_issue(ac + 1);
    if (a.n_heads > 2) q.act2 = ld_nc_issue(ac + 2);
    if (a.n_heads > 3) q.act3 = ld_nc_issue(ac + 3);
    q.lpo = ld_nc_issue(a.logp_old + row);
    q.adv = ld_nc_issue(a.adv + row);
    return q;
}

// Bits of columns g .. g + 7 that lie in the head window [lo, hi) (g = lo
// rounded down to 8, then steps of 8), and of those the ones the mask allows.
__device__ __forceinline__ uint32_t window8(int g, int lo, int hi) {
    uint32_t b = 0xFFu;
    if (lo > g) b &= 0xFFu << (lo - g);
    if (hi - g < 8) b &= (1u << (hi - g)) - 1u;
    return b;
}
__device__ __forceinline__ uint32_t mask8(uint32_t w0, uint32_t w1, int g) {
    return ((g < 32 ? w0 : w1) >> (g & 31)) & 0xFFu;
}

// Section 4, actor part of one minibatch row, from its logits in TMEM (this
// lane's columns from taddr, plus the head bias b3).  Per head, two passes
// over 8-column groups (loops not unrolled: the code runs once per row and
// tile): the maximum of the allowed logits, then the exp weights e_k (kept in
// scr, this thread's column of a [64][128] float array), their sum S and
// sum e_k (l_k - max), which gives the head's entropy log S - that / S.  Then
// the clipped surrogate on the normalised advantage and the entropy bonus,
// and d loss / d logits (0 at masked actions, beyond O and, when !live, in
// the whole row) written into row `row` of the BF16 operand dl [BM][KO].
__device__ __forceinline__ ActorRow actor_row_tmem(const FbArgs& a, const RowIn& in, bool live, uint32_t taddr,
                                                   const float* b3, float* scr, uint8_t* dl, int row, int KT,
                                                   float mean, float inv_std, float inv_n) {
    Head4 lse, ent_h, rS;
    float logp = 0.0f, ent = 0.0f;
    for (int h = 0; h < a.n_heads; ++h) {
        const int lo = h * a.head, hi = lo + a.head, act = lo + in.act(h);
        float m = -FLT_MAX;
#pragma unroll 1
        for (int g = lo & ~7; g < hi; g += 8) {
            float v[8];
            tmem_ld8(taddr + (uint32_t)g, v);
            const uint32_t vb = window8(g, lo, hi) & mask8(in.w0, in.w1, g);
#pragma unroll
            for (int j = 0; j < 8; ++j) m = ((vb >> j) & 1u) ? fmaxf(m, v[j] + b3[g + j]) : m;
        }
        float S = 0.0f, T = 0.0f, la = 0.0f;
#pragma unroll 1
        for (int g = lo & ~7; g < hi; g += 8) {
            float v[8];
            tmem_ld8(taddr + (uint32_t)g, v);
            const uint32_t wb = window8(g, lo, hi), vb = wb & mask8(in.w0, in.w1, g);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float d = v[j] + b3[g + j] - m;
                const float e = ((vb >> j) & 1u) ? expf(d) : 0.0f;
                S += e;
                T += e * d;
                la = g + j == act ? d : la;
                if ((wb >> j) & 1u) scr[(g + j) * 128] = e;
            }
        }
        const float logS = logf(S), inv_S = 1.0f / S;
        logp += la - logS;
        const float Hh = logS - T * inv_S;
        ent += Hh;
        lse.set(h, m + logS);
        ent_h.set(h, Hh);
        rS.set(h, inv_S);
    }
    ActorRow st;
    const float lpo = in.lpo;
    const float ratio = expf(logp - lpo);
    const float an = (in.adv - mean) * inv_std;
    const float cr = fminf(fmaxf(ratio, 1.0f - a.clip), 1.0f + a.clip);
    const float s1 = ratio * an, s2 = cr * an;
    st.pg = -fminf(s1, s2);
    const bool inside = ratio > 1.0f - a.clip && ratio < 1.0f + a.clip;
    const float dratio = (s1 <= s2 || inside) ? -an : 0.0f;
    const float dlogp = live ? dratio * ratio * inv_n : 0.0f;
    st.clip = fabsf(ratio - 1.0f) > a.clip ? 1.0f : 0.0f;
    st.kl = lpo - logp;
    st.ent = ent;
    const float ec = live ? a.ent_coef * inv_n : 0.0f;
    for (int h = 0; h < a.n_heads; ++h) {
        const int lo = h * a.head, hi = lo + a.head, act = lo + in.act(h);
        const float o = lse.get(h), Hh = ent_h.get(h), inv_S = rS.get(h);
#pragma unroll 1
        for (int g = lo & ~7; g < hi; g += 8) {
            float v[8];
            tmem_ld8(taddr + (uint32_t)g, v);
            const uint32_t wb = window8(g, lo, hi), vb = wb & mask8(in.w0, in.w1, g);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = g + j;
                const float pk = scr[(((wb >> j) & 1u) ? k : 0) * 128] * inv_S;
                const float lp = v[j] + b3[k] - o;
                const float gk = dlogp * ((k == act ? 1.0f : 0.0f) - pk) + ec * pk * (lp + Hh);
                if ((wb >> j) & 1u) scr[k * 128] = ((vb >> j) & 1u) ? gk : 0.0f;
            }
        }
    }
    // gradient row -> BF16 operand (columns O .. KT - 1 zero)
    const int O = a.O;
#pragma unroll 1
    for (int c8 = 0; c8 < KT; c8 += 8) {
        float f[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) f[j] = c8 + j < O ? scr[(c8 + j) * 128] : 0.0f;
        st_shared_v4(dl + sw128_offset(row, c8, BM), pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]),
                     pack2(f[6], f[7]));
    }
    return st;
}

// The same row for at most 32 logits, in registers: one TMEM load of the 32
// logit columns, unrolled passes over the 8-column groups that hold logits
// (a uniform guard skips the others), l - max kept in place per head, and
// exp as ex2 of the scaled argument (__expf: a few units in the last place,
// the same value in both passes, so the probabilities are e / S of the e that
// make up S).
__device__ __forceinline__ ActorRow actor_row_reg32(const FbArgs& a, const RowIn& in, bool live, uint32_t taddr,
                                                    const float* b3, uint8_t* dl, int row, float mean, float inv_std,
                                                    float inv_n) {
    float l[32];
    tmem_ld32(taddr, l);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 b = *reinterpret_cast<const float4*>(b3 + 4 * q);
        l[4 * q] += b.x; l[4 * q + 1] += b.y; l[4 * q + 2] += b.z; l[4 * q + 3] += b.w;
    }
    const int ng = (a.O + 7) >> 3;                   // groups holding logits
    Head4 lS, ent_h, rS;
    float logp = 0.0f, ent = 0.0f;
#pragma unroll 1
    for (int h = 0; h < a.n_heads; ++h) {
        const int lo = h * a.head, hi = lo + a.head, act = lo + in.act(h);
        const uint32_t win = (hi >= 32 ? 0xFFFFFFFFu : (1u << hi) - 1u) & ~((1u << lo) - 1u);
        const uint32_t vb = win & in.w0;
        float m = -FLT_MAX;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < ng) {
#pragma unroll
                for (int j = 8 * q; j < 8 * q + 8; ++j) m = ((vb >> j) & 1u) ? fmaxf(m, l[j]) : m;
            }
        float S = 0.0f, T = 0.0f, la = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < ng) {
#pragma unroll
                for (int j = 8 * q; j < 8 * q + 8; ++j) {
                    const float d = l[j] - m;
                    l[j] = ((win >> j) & 1u) ? d : l[j];
                    const float e = ((vb >> j) & 1u) ? __expf(d) : 0.0f;
                    S += e;
                    T += e * d;
                    la = j == act ? d : la;
                }
            }
        const float logS = logf(S), inv_S = 1.0f / S;
        logp += la - logS;
        const float Hh = logS - T * inv_S;
        ent += Hh;
        lS.set(h, logS);
        ent_h.set(h, Hh);
        rS.set(h, inv_S);
    }
    ActorRow st;
    const float lpo = in.lpo;
    const float ratio = expf(logp - lpo);
    const float an = (in.adv - mean) * inv_std;
    const float cr = fminf(fmaxf(ratio, 1.0f - a.clip), 1.0f + a.clip);
    const float s1 = ratio * an, s2 = cr * an;
    st.pg = -fminf(s1, s2);
    const bool inside = ratio > 1.0f - a.clip && ratio < 1.0f + a.clip;
    const float dratio = (s1 <= s2 || inside) ? -an : 0.0f;
    const float dlogp = live ? dratio * ratio * inv_n : 0.0f;
    st.clip = fabsf(ratio - 1.0f) > a.clip ? 1.0f : 0.0f;
    st.kl = lpo - logp;
    st.ent = ent;
    const float ec = live ? a.ent_coef * inv_n : 0.0f;
    // d loss / d logits in place of l - max (0 at masked actions and beyond O)
#pragma unroll 1
    for (int h = 0; h < a.n_heads; ++h) {
        const int lo = h * a.head, hi = lo + a.head, act = lo + in.act(h);
        const uint32_t win = (hi >= 32 ? 0xFFFFFFFFu : (1u << hi) - 1u) & ~((1u << lo) - 1u);
        const uint32_t vb = win & in.w0;
        const float logS = lS.get(h), Hh = ent_h.get(h), inv_S = rS.get(h);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < ng) {
#pragma unroll
                for (int j = 8 * q; j < 8 * q + 8; ++j) {
                    const float pk = (((vb >> j) & 1u) ? __expf(l[j]) : 0.0f) * inv_S;
                    const float gk = dlogp * ((j == act ? 1.0f : 0.0f) - pk) + ec * pk * (l[j] - logS + Hh);
                    l[j] = ((win >> j) & 1u) ? (((vb >> j) & 1u) ? gk : 0.0f) : l[j];
                }
            }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) l[j] = j < a.O ? l[j] : 0.0f;
    // gradient row -> BF16 operand
#pragma unroll
    for (int c8 = 0; c8 < 32; c8 += 8)
        st_shared_v4(dl + sw128_offset(row, c8, BM), pack2(l[c8], l[c8 + 1]), pack2(l[c8 + 2], l[c8 + 3]),
                     pack2(l[c8 + 4], l[c8 + 5]), pack2(l[c8 + 6], l[c8 + 7]));
    return st;
}

template <int KT>
__global__ void __launch_bounds__(BT, 1) ppo_bf16_kernel(BfPpoArgs P) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ uint32_t src_rows[2][BM];      // rollout rows of this tile and of the next
    __shared__ float red[6][BT / 32];
    const FbArgs& a = P.f;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const PpoSmem L = ppo_smem();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int row = quarter * 32 + lane;             // TMEM lane of this thread
    const bool actor = (int)blockIdx.x < P.n_actor;
    const int role_cta = actor ? (int)blockIdx.x : (int)blockIdx.x - P.n_actor;
    const int role_ctas = actor ? P.n_actor : (int)gridDim.x - P.n_actor;
    const int I = a.in_dim, O = a.O;
    const NetOffsets off = net_offsets(I, HID, O);
    const float* w = a.weights;
    float* bias = (float*)(smem + L.bias);           // [0,128) b1|c1, [128,256) b2|c2, [256,320) b3|c3, [320,448) V3
    float* dv_s = bias + 448;                        // [BM] critic: d loss / d value per row
    float* v3r = bias + 576;                         // [HID] critic: V3 rounded to BF16 (the value head's operand)
    float* vpart = bias + 704;                       // [2][BM] critic: the two halves of each row's value

    // weights -> BF16 operands (row n of a B operand = output unit n)
    const size_t oW1 = actor ? off.W1 : off.V1, oW2 = actor ? off.W2 : off.V2;
    pack_operand(smem + L.w1, HID, KX, [&](int n, int k) { return k < I ? __ldg(w + oW1 + (size_t)k * HID + n) : 0.0f; });
    pack_operand(smem + L.w2, HID, HID, [&](int n, int k) { return __ldg(w + oW2 + (size_t)k * HID + n); });
    if (actor)
        pack_operand(smem + L.w3, KO, HID, [&](int n, int k) { return n < O ? __ldg(w + off.W3 + (size_t)k * O + n) : 0.0f; });
    else
        for (int k = tid; k < HID; k += BT) v3r[k] = __bfloat162float(__float2bfloat16_rn(w[off.V3 + k]));
    for (int k = tid; k < 448; k += BT) {
        float v = 0.0f;
        if (k < HID) v = w[(actor ? off.b1 : off.c1) + k];
        else if (k < 2 * HID) v = w[(actor ? off.b2 : off.c2) + k - HID];
        else if (k < 2 * HID + KO) v = actor ? (k - 2 * HID < O ? w[off.b3 + k - 2 * HID] : 0.0f) : (k == 2 * HID ? w[off.c3] : 0.0f);
        else if (!actor && k >= 320) v = w[off.V3 + k - 320];
        bias[k] = v;
    }
    for (int k = tid; k < BM * 64 * 2 / 16; k += BT) st_shared_v4(smem + L.ones + k * 16, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    for (int k = tid; k < 16 * BM * 2 / 16; k += BT) st_shared_v4(smem + L.dv + k * 16, 0u, 0u, 0u, 0u);
    // columns of x beyond the inputs and the ones column, and of dL beyond the
    // logits in registers, stay zero for every tile
    for (int k = tid; k < BM * KX * 2 / 16; k += BT) st_shared_v4(smem + L.x + k * 16, 0u, 0u, 0u, 0u);
    for (int k = tid; k < BM * KO * 2 / 16; k += BT) st_shared_v4(smem + L.dl + k * 16, 0u, 0u, 0u, 0u);
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, TMEM_COLS);
    sync_for_mma();
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t sw1 = smem_u32(smem + L.w1), sw2 = smem_u32(smem + L.w2), sw3 = smem_u32(smem + L.w3);
    const uint32_t sx = smem_u32(smem + L.x), sh1 = smem_u32(smem + L.h1), sh2 = smem_u32(smem + L.h2);
    const uint32_t sdl = smem_u32(smem + L.dl), sdz2 = smem_u32(smem + L.dz2), sones = smem_u32(smem + L.ones);
    const uint32_t sdv = smem_u32(smem + L.dv);

    // advantage moments over the minibatch (or over the union of the ranks'
    // minibatches, when given: count, sum, sum of squares)
    const double nrows_mb = a.moments ? a.moments[0] : (double)a.mb.count;
    const double m1 = a.moments ? a.moments[1] : a.stats[ST_ADV_SUM];
    const double m2 = a.moments ? a.moments[2] : a.stats[ST_ADV_SQ];
    const float mean = (float)(m1 / nrows_mb);
    const float var = (float)fmax(m2 / nrows_mb - (m1 / nrows_mb) * (m1 / nrows_mb), 0.0);
    const float inv_std = 1.0f / (sqrtf(var) + 1e-8f);
    const float inv_n = 1.0f / (float)nrows_mb;

    float acc_st[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};   // pg, vf, ent, clip, kl of this thread's rows
    float dc3_part = 0.0f;                               // critic: sum of this thread's rows' BF16 dv
    uint32_t phase = 0;
    bool ok = true, first = true, pending = false;
    const int n_tiles = (a.mb.count + BM - 1) / BM;
    // The gathered input rows go in a row per warp instruction (lane k: column
    // k), so each load touches one or two cache lines.  With inputs and the
    // ones column in 32 columns, the next tile's are loaded into registers
    // during the current one: in the actor by every warp (16 rows each), in
    // the critic by the second warpgroup (32 rows per warp); otherwise every
    // warp gathers 16 rows at the tile's start.
    constexpr int RPW = BM / 4, RPW8 = BM / (BT / 32);
    const bool x_all = actor;                         // loaders: all warps, or the second warpgroup
    const int x_rows = x_all ? RPW8 : RPW, x_r0 = x_all ? warp * RPW8 : quarter * RPW;
    const int xcols = (I / 8 + 1) * 8;               // columns written: inputs, the ones column, zeros
    const bool pf = I + 1 <= 32;
    uint32_t* rows_cur = src_rows[0];
    uint32_t* rows_nxt = src_rows[1];
    float xr[RPW];
    auto load_rows = [&](int t, uint32_t* dst) {
        if (tid < BM) {
            const int j = t * BM + tid;
            dst[tid] = (t < n_tiles && j < a.mb.count) ? (a.rows ? a.rows[j] : mb_row(a.mb, j)) : 0u;
        }
    };
    auto x_at = [&](const uint32_t* rr, int r, int nr, int k) {
        float v = (r < nr && k == I) ? 1.0f : 0.0f;
        if (r < nr && k < I) v = ld_nc_issue(a.x + (size_t)rr[r] * I + k);
        return v;
    };
    auto put_x = [&](int r, int k, float v) {   // lanes k, k + 1 -> one BF16 pair
        const float nx = __shfl_down_sync(0xFFFFFFFFu, v, 1);
        if ((lane & 1) == 0 && k < xcols) st_shared_u32(smem + L.x + sw128_offset(r, k, BM), pack2(v, nx));
    };
    auto load_x = [&](int t, const uint32_t* rr) {   // a loading warp's rows
        const int nr = t < n_tiles ? min(BM, a.mb.count - t * BM) : 0;
#pragma unroll
        for (int q = 0; q < RPW; ++q)
            if (q < x_rows) xr[q] = x_at(rr, x_r0 + q, nr, lane);
    };
    auto store_x = [&]() {   // the shuffles first, then the stores
        float nx[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q)
            if (q < x_rows) nx[q] = __shfl_down_sync(0xFFFFFFFFu, xr[q], 1);
        if ((lane & 1) == 0 && lane < xcols) {
#pragma unroll
            for (int q = 0; q < RPW; ++q)
                if (q < x_rows) st_shared_u32(smem + L.x + sw128_offset(x_r0 + q, lane, BM), pack2(xr[q], nx[q]));
        }
    };
    // this thread's row's loss inputs, for the tile whose rows are in rr
    // (loaded a tile ahead with the inputs; used after the forward pass)
    RowIn rin_nx{0xFFFFFFFFu, 0xFFFFFFFFu, 0, 0, 0, 0, 0.0f, 0.0f};
    float vo_nx = 0.0f, ret_nx = 0.0f;
    auto load_rin = [&](int t, const uint32_t* rr) {   // first warpgroup
        const int nr = t < n_tiles ? min(BM, a.mb.count - t * BM) : 0;
        if (half == 0 && row < nr) {
            const uint32_t src = rr[row];
            if (actor) rin_nx = load_row_in(a, src, KT > 32);
            else { vo_nx = ld_nc_issue(a.v_old + src); ret_nx = ld_nc_issue(a.ret + src); }
        }
    };
    // The next tile's inputs and loss inputs (first warpgroup), loaded while
    // the loading warps would otherwise wait: the actor's during its second
    // product, the critic's as thread 0 starts issuing the tile's last group
    // of products.  (The proxy fence ahead of a product waits for loads in
    // flight; of the placements measured, these gave the shortest update.)
    // rr: the row table of tile t (loaded and visible to every thread).
    auto prefetch = [&](int t, const uint32_t* rr) {
        if (pf) {
            if (x_all || half) load_x(t, rr);
            if (half == 0) load_rin(t, rr);
        }
        __syncwarp();   // converged again before any warp-collective TMEM access
    };
    // Two tiles ahead, the second warpgroup (thread 128 + i: the tile's row i)
    // reads the row table and asks L2 for the lines of that row's inputs and
    // loss inputs, so that the loads a tile later hit L2 rather than HBM.
    auto prefetch_l2_rows = [&](int t) {
        const int j = t * BM + (tid - BM);
        if (half == 1 && a.rows && t < n_tiles && j < a.mb.count) {
            const uint32_t r = a.rows[j];
            const float* xr0 = a.x + (size_t)r * I;
            prefetch_l2(xr0);
            prefetch_l2(xr0 + I - 1);
            if (actor) {
                if (a.W) prefetch_l2(a.mask + (size_t)r * a.W);
                prefetch_l2(a.act + (size_t)r * a.n_heads);
                prefetch_l2(a.logp_old + r);
                prefetch_l2(a.adv + r);
            } else {
                prefetch_l2(a.v_old + r);
                prefetch_l2(a.ret + r);
            }
        }
    };
    if (pf && role_cta < n_tiles) {
        prefetch_l2_rows(role_cta + role_ctas);
        load_rows(role_cta, rows_cur);
        __syncthreads();
        prefetch(role_cta, rows_cur);
    }
    for (int tile = role_cta; tile < n_tiles; tile += role_ctas) {
        const int j0 = tile * BM;
        const int nrows = min(BM, a.mb.count - j0);
        // the previous tile's last products read x, h1, h2, dL and dZ2: wait before overwriting them
        if (pending) {
            if (!(ok = wait_mma(&bar, phase))) break;
            pending = false;
        }
        if (pf) {
            if (x_all || half) store_x();
        } else {
            load_rows(tile, rows_cur);
            __syncthreads();
            // gathered rollout inputs -> x operand: inputs, then 1 (the bias column)
            for (int q = 0; q < RPW8; ++q)
                for (int c0 = 0; c0 < KX; c0 += 32)
                    put_x(warp * RPW8 + q, c0 + lane, x_at(rows_cur, warp * RPW8 + q, nrows, c0 + lane));
            load_rin(tile, rows_cur);
        }
        const RowIn rin = rin_nx;
        const float v_old = vo_nx, ret = ret_nx;
        sync_for_mma();
        // layer 1
        if (tid == 0) {
            chain<KX / 16, K_MAJ, BM, K_MAJ, HID>(tmem + C_SLOT, idesc_bf16(BM, HID), false, kdesc(sx), kdesc(sw1));
            mma_commit(&bar);
        }
        if (pf) load_rows(tile + role_ctas, rows_nxt);   // visible after the next barrier
        if (!(ok = wait_mma(&bar, phase))) break;
        relu_epilogue64(lane_base + C_SLOT + half * 64, bias + half * 64, smem + L.h1, row, half * 64);
        sync_for_mma();
        // layer 2
        if (tid == 0) {
            chain<HID / 16, K_MAJ, BM, K_MAJ, HID>(tmem + C_SLOT, idesc_bf16(BM, HID), false, kdesc(sh1), kdesc(sw2));
            mma_commit(&bar);
        }
        if (actor) prefetch(tile + role_ctas, rows_nxt);
        if (!(ok = wait_mma(&bar, phase))) break;
        if (actor) {
            relu_epilogue64(lane_base + C_SLOT + half * 64, bias + HID + half * 64, smem + L.h2, row, half * 64);
            sync_for_mma();
            // head: logits = H2 W3
            if (tid == 0) {
                chain<HID / 16, K_MAJ, BM, K_MAJ, KO>(tmem + C_SLOT, idesc_bf16(BM, (O + 15) & ~15), false, kdesc(sh2),
                                                       kdesc(sw3));
                mma_commit(&bar);
            }
            if (!(ok = wait_mma(&bar, phase))) break;
            if (pf) prefetch_l2_rows(tile + 2 * role_ctas);
            if (half == 0) {
                // the loss and d loss / d logits of this thread's row
                const bool live = row < nrows;
                ActorRow s;
                if constexpr (KT == 32)
                    s = actor_row_reg32(a, rin, live, lane_base + C_SLOT, bias + 2 * HID, smem + L.dl, row, mean,
                                        inv_std, inv_n);
                else
                    // scratch: the dZ2 buffer, free from the last tile's weight-gradient
                    // products to this tile's first mask epilogue
                    s = actor_row_tmem(a, rin, live, lane_base + C_SLOT, bias + 2 * HID,
                                       reinterpret_cast<float*>(smem + L.dz2) + row, smem + L.dl, row, KT, mean,
                                       inv_std, inv_n);
                if (live) { acc_st[0] += s.pg; acc_st[2] += s.ent; acc_st[3] += s.clip; acc_st[4] += s.kl; }
            }
            sync_for_mma();
            if (tid == 0) {
                // dZ2 (before the mask) = dL W3^T, committed alone: the mask epilogue waits only for it
                chain<KT / 16, K_MAJ, BM, MN_MAJ, KO>(tmem + C_SLOT, idesc_bf16(BM, HID) | TB, false, kdesc(sdl),
                                                       mndesc<KO>(sw3));
                mma_commit(&bar);
                // dW3 += H2^T dL;  db3 (every lane) += 1^T dL: done by the next commit
                chain<BM / 16, MN_MAJ, BM, MN_MAJ, BM>(tmem + C_W3, idesc_bf16(BM, KO) | TA | TB, !first,
                                                        mndesc<BM>(sh2), mndesc<BM>(sdl));
                chain<BM / 16, K_ONE, BM, MN_MAJ, BM>(tmem + C_B3, idesc_bf16(BM, KO) | TB, !first, kdesc(sones),
                                                       mndesc<BM>(sdl));
            }
            if (!(ok = wait_mma(&bar, phase))) break;
            mask_epilogue64(lane_base + C_SLOT + half * 64, smem + L.h2, smem + L.dz2, row, half * 64);
            sync_for_mma();
            if (tid == 0) {
                // dZ1 (before the mask) = dZ2 W2^T; this commit also covers dW3 and db3,
                // which read the h2 buffer the mask epilogue then overwrites
                chain<HID / 16, K_MAJ, BM, MN_MAJ, HID>(tmem + C_SLOT, idesc_bf16(BM, HID) | TB, false, kdesc(sdz2),
                                                         mndesc<HID>(sw2));
                mma_commit(&bar);
                // dW2^T | db2 += dZ2^T [H1 | 1] (the all-ones panel follows H1): done by the
                // tile's last commit
                chain<BM / 16, MN_MAJ, BM, MN_MAJ, BM>(tmem + C_W2, idesc_bf16(BM, HID + 16) | TA | TB, !first,
                                                        mndesc<BM>(sdz2), mndesc<BM>(sh1));
            }
        } else {
            // G2, and the value head on the CUDA cores: each thread's half of the
            // row's products with the BF16 V3 entries, summed over the halves
            const float vp = relu_epilogue64(lane_base + C_SLOT + half * 64, bias + HID + half * 64, smem + L.h2, row,
                                             half * 64, v3r + half * 64);
            vpart[half * BM + row] = vp;
            sync_for_mma();
            if (half == 0) {
                float dv = 0.0f;
                if (row < nrows) {
                    // Section 4 clipped value loss, 0.5 max((v - R)^2, (v_clipped - R)^2)
                    const float v = (vpart[row] + vpart[BM + row]) + bias[2 * HID], vo = v_old, R = ret;
                    const float dvv = v - vo;
                    const float vc = vo + fminf(fmaxf(dvv, -a.vclip), a.vclip);
                    const float la = (v - R) * (v - R), lb = (vc - R) * (vc - R);
                    acc_st[1] += 0.5f * fmaxf(la, lb);
                    dv = (la >= lb ? (v - R) : ((vc - R) * (fabsf(dvv) < a.vclip ? 1.0f : 0.0f))) * a.vf_coef * inv_n;
                }
                dv_s[row] = dv;
                const __nv_bfloat16 dvb = __float2bfloat16_rn(dv);
                *reinterpret_cast<__nv_bfloat16*>(smem + L.dv + sw128_offset(0, row, 16)) = dvb;
                dc3_part += __bfloat162float(dvb);       // dc3: the sum of the BF16 operand dv
            }
            __syncthreads();
            // dY2 = dv V3^T, masked by [g2 > 0] (G2 is in the h2 buffer)
            {
                const float dv = dv_s[row];
                const __nv_bfloat162 zero = __floats2bfloat162_rn(0.0f, 0.0f);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int col = half * 64 + q * 8;
                    const uint4 hq = *reinterpret_cast<const uint4*>(smem + L.h2 + sw128_offset(row, col, BM));
                    const uint32_t hw[4] = {hq.x, hq.y, hq.z, hq.w};
                    uint32_t wv[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float* v3 = bias + 320 + col + 2 * j;
                        wv[j] = bf2_bits(__hmul2(__floats2bfloat162_rn(dv * v3[0], dv * v3[1]), __hgt2(bits_bf2(hw[j]), zero)));
                    }
                    st_shared_v4(smem + L.dz2 + sw128_offset(row, col, BM), wv[0], wv[1], wv[2], wv[3]);
                }
            }
            sync_for_mma();
            prefetch(tile + role_ctas, rows_nxt);
            if (pf) prefetch_l2_rows(tile + 2 * role_ctas);
            if (tid == 0) {
                // dY1 (before the mask) = dY2 V2^T and dV3 += G2^T dv, committed
                // together: the mask epilogue overwrites G2 in the h2 buffer
                chain<HID / 16, K_MAJ, BM, MN_MAJ, HID>(tmem + C_SLOT, idesc_bf16(BM, HID) | TB, false, kdesc(sdz2),
                                                         mndesc<HID>(sw2));
                chain<BM / 16, MN_MAJ, BM, K_MAJ, 16>(tmem + C_V3, idesc_bf16(BM, 16) | TA, !first, mndesc<BM>(sh2),
                                                       kdesc(sdv));
                mma_commit(&bar);
                // dV2^T | dc2 += dY2^T [G1 | 1]: done by the tile's last commit
                chain<BM / 16, MN_MAJ, BM, MN_MAJ, BM>(tmem + C_W2, idesc_bf16(BM, HID + 16) | TA | TB, !first,
                                                        mndesc<BM>(sdz2), mndesc<BM>(sh1));
            }
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        // first-layer gradient of the pre-activation: dZ1 / dY1 into the h2 buffer
        mask_epilogue64(lane_base + C_SLOT + half * 64, smem + L.h1, smem + L.h2, row, half * 64);
        sync_for_mma();
        if (tid == 0) {
            // dW1^T += dZ1^T X (column I of X is 1: the first-layer bias gradient)
            chain<BM / 16, MN_MAJ, BM, MN_MAJ, BM>(tmem + C_W1T, idesc_bf16(BM, KX) | TA | TB, !first, mndesc<BM>(sh2),
                                                    mndesc<BM>(sx));
            mma_commit(&bar);
        }
        pending = true;
        first = false;
        uint32_t* tmp = rows_cur;
        rows_cur = rows_nxt;
        rows_nxt = tmp;
    }
    if (ok && pending) ok = wait_mma(&bar, phase);
    if (ok) {
        float* out = P.partial + (size_t)blockIdx.x * BM * PC;
        const int c0 = half == 0 ? 0 : 6, c1 = half == 0 ? 6 : PC / 32;
        for (int ch = c0; ch < c1; ++ch) {
            float v[32];
            tmem_ld32(lane_base + ch * 32, v);
            float4* dst = reinterpret_cast<float4*>(out + (size_t)row * PC + ch * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
    } else {
        // a wait gave up: give the tensor core one more bounded chance to finish before freeing TMEM
        mbar_wait(&bar, phase, 200000000LL);
    }
    // loss statistics of this CTA's rows, and the critic's dc3
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        float v = q < 5 ? acc_st[q] : dc3_part;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if (lane == 0) red[q][warp] = v;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 5) {
        double s = 0.0;
        for (int k = 0; k < BT / 32; ++k) s += red[tid][k];
        if (s != 0.0) atomicAdd(&a.stats[ST_PG + tid], s);
    }
    if (tid == 5 && ok && !actor) {
        // after the accumulator dump above (ordered by the barrier): dc3 of this CTA
        float s = 0.0f;
        for (int k = 0; k < BT / 32; ++k) s += red[5][k];
        P.partial[(size_t)blockIdx.x * BM * PC + C_C3] = s;
    }
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// Sums the CTAs' accumulators into the gradient vector (padding = 0).
__global__ void ppo_bf16_reduce_kernel(const float* __restrict__ partial, int n_actor, int n_critic, int I, int O,
                                       float* __restrict__ grad) {
    // Items [0, 2 BM PC): one (role, lane, column) of the CTAs' partial rows,
    // consecutive items on consecutive columns (coalesced reads), summed over
    // the role's CTAs in CTA order into the parameter that column holds.
    // Items past that: the parameter vector's padding, written 0.
    const NetOffsets o = net_offsets(I, HID, O);
    constexpr int per_role = BM * PC;
    const size_t n_items = 2 * (size_t)per_role + o.total;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_items; e += (size_t)gridDim.x * blockDim.x) {
        if (e >= 2 * (size_t)per_role) {
            const size_t p = e - 2 * (size_t)per_role;
            auto in = [&](size_t base, size_t n) { return p >= base && p < base + n; };
            const bool used = in(o.W1, (size_t)I * HID) || in(o.b1, HID) || in(o.W2, HID * HID) || in(o.b2, HID) ||
                              in(o.W3, (size_t)HID * O) || in(o.b3, O) || in(o.V1, (size_t)I * HID) ||
                              in(o.c1, HID) || in(o.V2, HID * HID) || in(o.c2, HID) || in(o.V3, HID) || in(o.c3, 1);
            if (!used) grad[p] = 0.0f;
            continue;
        }
        const bool act = e < (size_t)per_role;
        const int le = (int)(act ? e : e - per_role);
        const int lane = le / PC, col = le % PC;
        long long p = -1;
        if (col < I) p = (long long)(act ? o.W1 : o.V1) + (long long)col * HID + lane;
        else if (col == I) p = (long long)(act ? o.b1 : o.c1) + lane;
        else if (col >= (int)C_W2 && col < (int)C_W2 + HID) p = (long long)(act ? o.W2 : o.V2) + (long long)(col - C_W2) * HID + lane;
        else if (col == (int)(act ? C_B2 : C_C2)) p = (long long)(act ? o.b2 : o.c2) + lane;
        else if (act && col >= (int)C_W3 && col < (int)C_W3 + O) p = (long long)o.W3 + (long long)lane * O + (col - C_W3);
        else if (act && col >= (int)C_B3 && col < (int)C_B3 + O && lane == 0) p = (long long)o.b3 + (col - C_B3);
        else if (!act && col == (int)C_V3) p = (long long)o.V3 + lane;
        else if (!act && col == (int)C_C3 && lane == 0) p = (long long)o.c3;
        if (p < 0) continue;
        const int c0 = act ? 0 : n_actor, c1 = act ? n_actor : n_actor + n_critic;
        float sum = 0.0f;
#pragma unroll 8
        for (int c = c0; c < c1; ++c) sum += partial[(size_t)c * per_role + le];
        grad[p] = sum;
    }
}

int sm_count() {
    const int n = device_sms();
    return n < 2 ? 2 : n;
}

}  // namespace

ej_status bf16_grad_shape(int in_dim, int H, int O, int n_heads, int W) {
    if (H != HID) return fail(EJ_ERR_UNSUPPORTED, "bf16 PPO: hidden must be %d", HID);
    if (in_dim + 1 > KX) return fail(EJ_ERR_UNSUPPORTED, "bf16 PPO: input width must be <= %d", KX - 1);
    if (O > KO) return fail(EJ_ERR_UNSUPPORTED, "bf16 PPO: at most %d logits", KO);
    if (n_heads < 1 || n_heads > 4) return fail(EJ_ERR_UNSUPPORTED, "bf16 PPO: 1 to 4 action heads");
    if (W > 2) return fail(EJ_ERR_UNSUPPORTED, "bf16 PPO: at most 2 mask words");
    return EJ_OK;
}

ej_status launch_ppo_bf16(const FbArgs& fa, float* partial, size_t partial_bytes, float* grad, cudaStream_t s) {
    ej_status st = bf16_grad_shape(fa.in_dim, fa.H, fa.O, fa.n_heads, fa.W);
    if (st != EJ_OK) return st;
    if (!fa.rows && (st = launch_adv_stats(fa.mb, fa.adv, fa.stats, s)) != EJ_OK) return st;
    const NetOffsets off = net_offsets(fa.in_dim, HID, fa.O);
    const int n_tiles = (fa.mb.count + BM - 1) / BM;
    if (n_tiles < 1) {
        if (cudaMemsetAsync(grad, 0, sizeof(float) * off.total, s) != cudaSuccess) return fail(EJ_ERR_CUDA, "memset failed");
        return EJ_OK;
    }
    // actor and critic CTAs (one per SM in all): the split with the shortest
    // longer role, a role with n CTAs taking ceil(tiles / n) rounds of its
    // tile cost
    const int sms = sm_count();
    int groups = 0;
    for (int h = 0; h < fa.n_heads; ++h) groups += (h * fa.head + fa.head + 7) / 8 - (h * fa.head) / 8;
    const double c_act = PPO_TILE + (fa.O <= 32 ? PPO_LOSS_REG : PPO_LOSS_GROUP * groups), c_cri = PPO_TILE;
    int n_act = 1, n_cri = 1;
    double best = 1e300;
    for (int na = 1; na < sms && na <= n_tiles; ++na) {
        const int nc = sms - na < n_tiles ? sms - na : n_tiles;
        const double t = fmax(c_act * ((n_tiles + na - 1) / na), c_cri * ((n_tiles + nc - 1) / nc));
        if (t < best) { best = t; n_act = na; n_cri = nc; }
    }
    if ((size_t)(n_act + n_cri) * BM * PC * sizeof(float) > partial_bytes)
        return fail(EJ_ERR_UNSUPPORTED, "bf16 PPO: workspace too small for %d CTAs", n_act + n_cri);
    const size_t smem = ppo_smem().total + 1024;
    static SmemOptIn opt_in[2];
    const int kt = fa.O <= 32 ? 0 : 1;
    st = opt_in[kt].ensure(kt == 0 ? (const void*)ppo_bf16_kernel<32> : (const void*)ppo_bf16_kernel<64>, smem);
    if (st != EJ_OK) return st;
    BfPpoArgs P;
    P.f = fa;
    P.partial = partial;
    P.n_actor = n_act;
    if (fa.rows) {
        st = launch_mb_rows_stats(fa.mb, fa.adv, fa.rows, fa.stats, s);
        if (st != EJ_OK) return st;
    }
    if (kt == 0) ppo_bf16_kernel<32><<<n_act + n_cri, BT, smem, s>>>(P);
    else ppo_bf16_kernel<64><<<n_act + n_cri, BT, smem, s>>>(P);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "bf16 PPO launch: %s", cudaGetErrorString(err));
    ppo_bf16_reduce_kernel<<<sm_count() * 4, 256, 0, s>>>(partial, n_act, n_cri, fa.in_dim, fa.O, grad);
    err = cudaGetLastError();
    if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "bf16 PPO reduce launch: %s", cudaGetErrorString(err));
    return EJ_OK;
}

int ppo_bf16_fault(int clear) {
    int v = 0;
    cudaMemcpyFromSymbol(&v, g_ej_fault, sizeof(int));
    if (clear) {
        const int z = 0;
        cudaMemcpyToSymbol(g_ej_fault, &z, sizeof(int));
    }
    return v;
}

}  // namespace ej
