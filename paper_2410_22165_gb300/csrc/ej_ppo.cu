// PPO update of Section 4 (Table 2: clip 0.2, value coefficient 0.25, value
// clip 10, entropy coefficient 0.1, GAE lambda 0.95), float32 on the CUDA
// cores: GAE, per-minibatch advantage normalisation, a fused tile kernel
// (forward, loss gradient, backward through the activations), a split-K
// weight-gradient kernel with its reduction, and Adam.
#include <cfloat>
#include <cmath>
#include <cstring>

#include "ej_internal.cuh"
#include "ej_policy.cuh"
#include "ej_ppo.cuh"

namespace ej {

namespace {

// ---------------------------------------------------------------- GAE
__global__ void gae_kernel(const float* __restrict__ rew, const float* __restrict__ value,
                           const uint8_t* __restrict__ done, int T, int rows, int per_env, float gamma,
                           float lam, float* __restrict__ adv, float* __restrict__ ret) {
    const int E = rows / per_env;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += gridDim.x * blockDim.x) {
        const int e = row / per_env;
        float next = 0.0f;
        for (int t = T - 1; t >= 0; --t) {
            const float nd = done[(size_t)t * E + e] ? 0.0f : 1.0f;
            const float v = value[(size_t)t * rows + row];
            const float vn = value[(size_t)(t + 1) * rows + row];
            const float delta = rew[(size_t)t * rows + row] + gamma * nd * vn - v;
            next = delta + gamma * lam * nd * next;
            adv[(size_t)t * rows + row] = next;
            ret[(size_t)t * rows + row] = next + v;
        }
    }
}

// ------------------------------------- minibatch advantage statistics
__global__ void adv_stats_kernel(MbDesc d, const float* __restrict__ adv, double* stats) {
    double s = 0.0, q = 0.0;
    mb_rows_strided(d, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, [&](int, uint32_t r) {
        const double a = adv[r];
        s += a;
        q += a * a;
    });
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        q += __shfl_xor_sync(0xFFFFFFFFu, q, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&stats[ST_ADV_SUM], s);
        atomicAdd(&stats[ST_ADV_SQ], q);
    }
}

// rows[j] = the rollout row at position lo + j of the minibatch permutation,
// and the advantage sums over those rows.
__global__ void mb_rows_stats_kernel(MbDesc d, const float* __restrict__ adv, uint32_t* __restrict__ rows,
                                     double* stats) {
    double s = 0.0, q = 0.0;
    mb_rows_strided(d, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, [&](int j, uint32_t r) {
        rows[j] = r;
        const double a = adv[r];
        s += a;
        q += a * a;
    });
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        q += __shfl_xor_sync(0xFFFFFFFFu, q, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&stats[ST_ADV_SUM], s);
        atomicAdd(&stats[ST_ADV_SQ], q);
    }
}

__global__ void zero_kernel(double* p, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) p[k] = 0.0;
}

// Maximum and sum over an aligned group of eight lanes (mask `gm`); the
// butterfly leaves the same value in every lane of the group.
__device__ __forceinline__ float group8_max(float v, unsigned gm) {
    v = fmaxf(v, __shfl_xor_sync(gm, v, 4, 8));
    v = fmaxf(v, __shfl_xor_sync(gm, v, 2, 8));
    return fmaxf(v, __shfl_xor_sync(gm, v, 1, 8));
}
__device__ __forceinline__ float group8_sum(float v, unsigned gm) {
    v += __shfl_xor_sync(gm, v, 4, 8);
    v += __shfl_xor_sync(gm, v, 2, 8);
    return v + __shfl_xor_sync(gm, v, 1, 8);
}

// ---------------------------------- fused forward + loss + backward-data
// 32-row tiles (thread tiles of 4 rows x 4 columns) and at most 80 registers
// a thread: three CTAs (24 warps) share an SM at hidden 128, two at 256.
constexpr int PTILE = 32;
// Per tile of PTILE (32) minibatch rows: gather the rollout rows, run actor and
// critic, form the gradient of the clipped PPO loss with respect to the
// logits and the value, and back-propagate it through the hidden layers.
// Every activation and activation gradient the weight gradients need is
// written to the workspace.
__global__ void __launch_bounds__(NTH, 3) fwd_bwd_kernel(FbArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int H = a.H, O = a.O, I = a.in_dim;
    const int ldx = a.in_pad, ldh = H + 4, ldo = ((O + 3) & ~3) + 4;
    float* xs = sm;                      // [PTILE][ldx]
    float* B0 = xs + PTILE * ldx;         // [PTILE][ldh]
    float* B1 = B0 + PTILE * ldh;
    float* B2 = B1 + PTILE * ldh;
    float* LG = B2 + PTILE * ldh;         // [PTILE][ldo]
    float* VAL = LG + PTILE * ldo;        // [PTILE]
    float* DV = VAL + PTILE;              // [PTILE]
    __shared__ float red[8][NTH / 32];
    const NetOffsets off = net_offsets(I, H, O);
    // advantage moments over the minibatch (or over the union of the ranks'
    // minibatches, when given: count, sum, sum of squares); per agent for
    // per-agent networks
    const double n_mb = a.moments ? a.moments[0] : (double)a.mb.count;
    const int tpa = (a.mb.count + PTILE - 1) / PTILE;     // tiles per agent (the minibatch's, shared networks)
    const int n_tiles = a.agents ? a.agents * tpa : tpa;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int agent = a.agents ? tile / tpa : 0;
        const int j0 = (a.agents ? tile % tpa : tile) * PTILE;   // position in the (agent's) minibatch
        const int nvalid = min(PTILE, a.mb.count - j0);
        const int base = agent * a.mb.count + j0;               // row of the per-row buffers
        const float* wa = a.weights + (size_t)agent * a.actor_stride;
        const float* wc = a.weights + (size_t)agent * a.critic_stride;
        const float* w3t = a.w3t + (size_t)agent * O * H;
        const float* w2t = a.w2t + (size_t)agent * H * H;
        const float* v2t = a.v2t + (a.critic_stride ? (size_t)agent * H * H : 0);
        double n = n_mb, m1, m2;
        if (a.agents) {
            n = (double)a.mb.count;
            m1 = a.agent_moments[2 * agent];
            m2 = a.agent_moments[2 * agent + 1];
        } else {
            m1 = a.moments ? a.moments[1] : a.stats[ST_ADV_SUM];
            m2 = a.moments ? a.moments[2] : a.stats[ST_ADV_SQ];
        }
        const float mean = (float)(m1 / n);
        const float var = (float)fmax(m2 / n - (m1 / n) * (m1 / n), 0.0);
        const float inv_std = 1.0f / (sqrtf(var) + 1e-8f);
        const float inv_n = 1.0f / (float)n;
        // the critic's loss: the mean over its own rows (a shared critic of
        // per-agent actors: over every agent's rows)
        const float inv_nc = (a.agents && !a.critic_stride) ? 1.0f / (float)(n * a.agents) : inv_n;
        // gather
        __shared__ uint32_t src_row[PTILE];
        if (threadIdx.x < PTILE) {
            const int j = j0 + threadIdx.x;
            src_row[threadIdx.x] = j < a.mb.count ? (a.agents ? mb_row(a.mb, j) * (uint32_t)a.agents + (uint32_t)agent
                                                              : mb_row(a.mb, j)) : 0u;
        }
        __syncthreads();
        tile_for<PTILE>(ldx, [&](int r, int k) {
            const bool in = r < nvalid && k < I;
            xs[r * ldx + k] = in ? a.x[(size_t)src_row[r] * I + k] : 0.0f;
        });
        __syncthreads();
        // actor forward
        dense_tile<PTILE, 4>(xs, ldx, I, wa + off.W1, wa + off.b1, H, B0, ldh, true);
        __syncthreads();
        dense_tile<PTILE, 4>(B0, ldh, H, wa + off.W2, wa + off.b2, H, B1, ldh, true);
        __syncthreads();
        head_tile<PTILE, 4>(B1, ldh, H, wa + off.W3, wa + off.b3, O, LG, ldo);
        __syncthreads();
        store_tile<PTILE>(xs, ldx, I, a.ws_x, base, nvalid);
        store_tile<PTILE>(B0, ldh, H, a.ws_h1, base, nvalid);
        store_tile<PTILE>(B1, ldh, H, a.ws_h2, base, nvalid);
        // loss gradient with respect to the logits: eight lanes per row, each
        // taking every eighth logit of a head; maxima and sums over the eight
        // lanes by butterflies (every lane ends with the same value)
        float pg = 0.0f, ent_sum = 0.0f, clipc = 0.0f, kl = 0.0f;
        static_assert(NTH == PTILE * 8, "eight lanes per row");
        if ((int)(threadIdx.x >> 3) < nvalid) {
            const int r = threadIdx.x >> 3, sub = threadIdx.x & 7;
            const unsigned gm = 0xFFu << (threadIdx.x & 24);
            const uint32_t row = src_row[r];
            float* l = LG + r * ldo;
            const uint32_t* mw = a.W ? a.mask + (size_t)row * a.W : nullptr;
            float logp = 0.0f;
            // per head: masked log-softmax, p
            for (int h = 0; h < a.n_heads; ++h) {
                float* lh = l + h * a.head;
                float m = -FLT_MAX;
                for (int k = sub; k < a.head; k += 8) {
                    const int bit = h * a.head + k;
                    if (!mw || ((mw[bit >> 5] >> (bit & 31)) & 1u)) m = fmaxf(m, lh[k]);
                }
                m = group8_max(m, gm);
                float S = 0.0f;
                for (int k = sub; k < a.head; k += 8) {
                    const int bit = h * a.head + k;
                    if (!mw || ((mw[bit >> 5] >> (bit & 31)) & 1u)) S += expf(lh[k] - m);
                }
                const float logS = logf(group8_sum(S, gm));
                const int act = a.act[(size_t)row * a.n_heads + h];
                logp += lh[act] - m - logS;
                __syncwarp(gm);     // lh[act] read by every lane before it is overwritten
                // keep log p in place (masked entries: +inf marker)
                float Hh = 0.0f;
                for (int k = sub; k < a.head; k += 8) {
                    const int bit = h * a.head + k;
                    const bool ok = !mw || ((mw[bit >> 5] >> (bit & 31)) & 1u);
                    const float lp = lh[k] - m - logS;
                    if (ok) Hh -= expf(lp) * lp;
                    lh[k] = ok ? lp : FLT_MAX;
                }
                Hh = group8_sum(Hh, gm);
                ent_sum += Hh;
                if (sub == 0) LG[r * ldo + O + (h & 3)] = Hh;   // per-head entropy (O is padded by at least 4)
            }
            const float lpo = a.logp_old[row];
            const float ratio = expf(logp - lpo);
            const float an = (a.adv[row] - mean) * inv_std;
            const float cr = fminf(fmaxf(ratio, 1.0f - a.clip), 1.0f + a.clip);
            const float s1 = ratio * an, s2 = cr * an;
            pg = -fminf(s1, s2);
            const bool inside = ratio > 1.0f - a.clip && ratio < 1.0f + a.clip;
            const float dratio = (s1 <= s2 || inside) ? -an : 0.0f;
            const float dlogp = dratio * ratio * inv_n;
            clipc = fabsf(ratio - 1.0f) > a.clip ? 1.0f : 0.0f;
            kl = lpo - logp;
            __syncwarp(gm);         // the entropies and every log p stored
            for (int h = 0; h < a.n_heads; ++h) {
                float* lh = l + h * a.head;
                const int act = a.act[(size_t)row * a.n_heads + h];
                const float Hh = LG[r * ldo + O + (h & 3)];
                for (int k = sub; k < a.head; k += 8) {
                    const float lp = lh[k];
                    float g = 0.0f;
                    if (lp != FLT_MAX) {
                        const float p = expf(lp);
                        g = dlogp * ((k == act ? 1.0f : 0.0f) - p) + a.ent_coef * inv_n * p * (lp + Hh);
                    }
                    lh[k] = g;
                }
            }
            if (sub != 0) pg = ent_sum = clipc = kl = 0.0f;   // each row counted once in the statistics
        }
        __syncthreads();
        store_tile<PTILE>(LG, ldo, O, a.ws_dl, base, nvalid);
        // dZ2 = (dL W3^T) * [h2 > 0]
        dense_tile<PTILE, 4>(LG, ldo, O, w3t, nullptr, H, B2, ldh, false);
        __syncthreads();
        mask_tile<PTILE>(B2, ldh, B1, H);
        __syncthreads();
        store_tile<PTILE>(B2, ldh, H, a.ws_dz2, base, nvalid);
        // dZ1 = (dZ2 W2^T) * [h1 > 0]
        dense_tile<PTILE, 4>(B2, ldh, H, w2t, nullptr, H, B1, ldh, false);
        __syncthreads();
        mask_tile<PTILE>(B1, ldh, B0, H);
        __syncthreads();
        store_tile<PTILE>(B1, ldh, H, a.ws_dz1, base, nvalid);
        // critic forward
        dense_tile<PTILE, 4>(xs, ldx, I, wc + off.V1, wc + off.c1, H, B0, ldh, true);
        __syncthreads();
        dense_tile<PTILE, 4>(B0, ldh, H, wc + off.V2, wc + off.c2, H, B1, ldh, true);
        __syncthreads();
        value_tile<PTILE>(B1, ldh, H, wc + off.V3, wc[off.c3], VAL);
        store_tile<PTILE>(B0, ldh, H, a.ws_g1, base, nvalid);
        store_tile<PTILE>(B1, ldh, H, a.ws_g2, base, nvalid);
        __syncthreads();
        // value-loss gradient (clipped value loss), one thread per row
        float vf = 0.0f;
        if (threadIdx.x < PTILE) {
            const int r = threadIdx.x;
            float dv = 0.0f;
            if (r < nvalid) {
                const uint32_t row = src_row[r];
                const float v = VAL[r], vo = a.v_old[row], R = a.ret[row];
                const float dvv = v - vo;
                const float vc = vo + fminf(fmaxf(dvv, -a.vclip), a.vclip);
                const float la = (v - R) * (v - R), lb = (vc - R) * (vc - R);
                vf = 0.5f * fmaxf(la, lb);
                dv = (la >= lb ? (v - R) : ((vc - R) * (fabsf(dvv) < a.vclip ? 1.0f : 0.0f))) * a.vf_coef * inv_nc;
                a.ws_dv[base + r] = dv;
            }
            DV[r] = dv;
        }
        __syncthreads();
        // dY2 = dv V3^T * [g2 > 0]
        tile_for<PTILE>(H >> 2, [&](int r, int c4) {
            const float4 g = *reinterpret_cast<const float4*>(B1 + r * ldh + 4 * c4);
            const float4 v3 = __ldg(reinterpret_cast<const float4*>(wc + off.V3 + 4 * c4));
            const float d = DV[r];
            float4 o;
            o.x = g.x > 0.0f ? d * v3.x : 0.0f;
            o.y = g.y > 0.0f ? d * v3.y : 0.0f;
            o.z = g.z > 0.0f ? d * v3.z : 0.0f;
            o.w = g.w > 0.0f ? d * v3.w : 0.0f;
            *reinterpret_cast<float4*>(B2 + r * ldh + 4 * c4) = o;
        });
        __syncthreads();
        store_tile<PTILE>(B2, ldh, H, a.ws_dy2, base, nvalid);
        dense_tile<PTILE, 4>(B2, ldh, H, v2t, nullptr, H, B1, ldh, false);
        __syncthreads();
        mask_tile<PTILE>(B1, ldh, B0, H);
        __syncthreads();
        store_tile<PTILE>(B1, ldh, H, a.ws_dy1, base, nvalid);
        // loss statistics
        float vals[5] = {pg, vf, ent_sum, clipc, kl};
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            float v = vals[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
            if (lane == 0) red[q][warp] = v;
        }
        __syncthreads();
        if (threadIdx.x < 5) {
            double s = 0.0;
            for (int k = 0; k < NTH / 32; ++k) s += red[threadIdx.x][k];
            atomicAdd(&a.stats[ST_PG + threadIdx.x], s);
        }
        __syncthreads();
    }
}

// --------------------------------------- split-K weight gradients
// Job q: G[m][n] = sum over minibatch rows of A[row][i] B[row][j], and the
// bias gradient sum of B[row][j]; rows split in chunks over blockIdx.x, the
// output in 128 x 128 tiles over blockIdx.z (hidden widths above 128).
//
// A block stages 32 rows of its A and B columns at a time in shared memory
// (cp.async, two stages: the next rows land while these are multiplied).  A
// thread owns an 8 x 8 block of G: rows {4 ti .. 4 ti + 3} and the same four
// rows a half-tile further, columns likewise (16-byte shared loads of
// consecutive threads are contiguous: no bank conflicts).  A tile narrower
// than 128 x 128 needs fewer threads; the block then runs S row slices
// (slice s takes rows s, s + S, ...) whose sums are added in slice order at
// the end.
constexpr int WG_ROWS = 32;
constexpr int WG_PITCH = WG_TILE + 4;
constexpr int WG_STAGE = 2 * WG_ROWS * WG_PITCH;        // floats of one stage (A and B)

struct WgShape {
    int tm, tn;      // 8 x 8 thread blocks over the tile's rows and columns
    int tp;          // threads of one slice (power of two >= tm * tn)
    int slices;      // NTH / tp
};

__host__ __device__ inline WgShape wg_shape(int m, int n) {
    WgShape w;
    const int mt = m < WG_TILE ? m : WG_TILE, nt = n < WG_TILE ? n : WG_TILE;
    w.tm = (mt + 7) / 8;
    w.tn = (nt + 7) / 8;
    w.tp = 1;
    while (w.tp < w.tm * w.tn) w.tp *= 2;
    w.slices = NTH / w.tp;
    return w;
}


__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// Copies rows [base, base + nr) of columns [c0, c0 + cols) of X (row pitch
// ld) into S[WG_ROWS][WG_PITCH].  The rest of S is left as it is: rows past nr
// are never read, and columns past cols only feed sums that are not stored.
__device__ __forceinline__ void wg_stage_copy(float* S, const float* __restrict__ X, int ld, int c0, int cols,
                                              int base, int nr, bool vec) {
    if (vec) {      // ld, c0 and cols multiples of 4, X 16-byte aligned
        const int cw = cols >> 2;
        for (int k = threadIdx.x; k < nr * cw; k += NTH) {
            const int r = k / cw, col = (k - r * cw) * 4;
            cp_async16(S + r * WG_PITCH + col, X + (size_t)(base + r) * ld + c0 + col);
        }
    } else {
        for (int k = threadIdx.x; k < nr * cols; k += NTH) {
            const int r = k / cols, col = k - r * cols;
            cp_async4(S + r * WG_PITCH + col, X + (size_t)(base + r) * ld + c0 + col);
        }
    }
}

__global__ void __launch_bounds__(NTH, 2) wgrad_kernel(WgJobs jobs, int rows, int chunks, size_t stride, int gmax,
                                                    float* __restrict__ partial) {
    extern __shared__ __align__(16) float wsm[];
    const WgJob jb = jobs.job[blockIdx.y];
    const int groups = jb.groups > 0 ? jb.groups : 1;
    const int grows = jb.groups > 0 ? jb.group_rows : rows;
    const int tiles_n = (jb.n + WG_TILE - 1) / WG_TILE, tiles_m = (jb.m + WG_TILE - 1) / WG_TILE;
    const int tiles = tiles_m * tiles_n;
    if ((int)blockIdx.z >= groups * tiles) return;
    const int g = (int)blockIdx.z / tiles, tz = (int)blockIdx.z % tiles;
    const int m0 = (tz / tiles_n) * WG_TILE, n0 = (tz % tiles_n) * WG_TILE;
    const int mt = min(WG_TILE, jb.m - m0), nt = min(WG_TILE, jb.n - n0);
    const WgShape sh = wg_shape(jb.m, jb.n);
    const int c = blockIdx.x;
    const int r0 = g * grows + (int)(((long long)grows * c) / chunks);
    const int r1 = g * grows + (int)(((long long)grows * (c + 1)) / chunks);
    const int slice = threadIdx.x / sh.tp, t = threadIdx.x % sh.tp;
    const bool active = t < sh.tm * sh.tn;
    const int ti = active ? t / sh.tn : 0, tj = active ? t % sh.tn : 0;
    const int hm = 4 * sh.tm, hn = 4 * sh.tn;        // the second four rows / columns
    const bool vec_a = (jb.lda & 3) == 0 && (m0 & 3) == 0 && (mt & 3) == 0 && ((uintptr_t)jb.A & 15) == 0;
    const bool vec_b = (jb.ldb & 3) == 0 && (n0 & 3) == 0 && (nt & 3) == 0 && ((uintptr_t)jb.B & 15) == 0;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
    float bsum = 0.0f;
    const bool bias_col = m0 == 0 && (int)threadIdx.x < nt;
    auto issue = [&](int stage, int base) {
        float* As = wsm + stage * WG_STAGE;
        const int nr = min(WG_ROWS, r1 - base);
        wg_stage_copy(As, jb.A, jb.lda, m0, mt, base, nr, vec_a);
        wg_stage_copy(As + WG_ROWS * WG_PITCH, jb.B, jb.ldb, n0, nt, base, nr, vec_b);
    };
    if (r0 < r1) issue(0, r0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    int it = 0;
    for (int base = r0; base < r1; base += WG_ROWS, ++it) {
        if (base + WG_ROWS < r1) issue((it + 1) & 1, base + WG_ROWS);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        const float* As = wsm + (it & 1) * WG_STAGE;
        const float* Bs = As + WG_ROWS * WG_PITCH;
        const int nr = min(WG_ROWS, r1 - base);
        if (active) {
            for (int r = slice; r < nr; r += sh.slices) {
                const float4 a0 = *reinterpret_cast<const float4*>(As + r * WG_PITCH + 4 * ti);
                const float4 a1 = *reinterpret_cast<const float4*>(As + r * WG_PITCH + hm + 4 * ti);
                const float4 b0 = *reinterpret_cast<const float4*>(Bs + r * WG_PITCH + 4 * tj);
                const float4 b1 = *reinterpret_cast<const float4*>(Bs + r * WG_PITCH + hn + 4 * tj);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int x = 0; x < 8; ++x)
#pragma unroll
                    for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
            }
        }
        if (bias_col) {
#pragma unroll
            for (int r8 = 0; r8 < WG_ROWS; r8 += 8) {
                float bt[8];        // loads issued together, then summed in row order
#pragma unroll
                for (int r = 0; r < 8; ++r) bt[r] = Bs[(r8 + r) * WG_PITCH + threadIdx.x];
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    if (r8 + r < nr) bsum += bt[r];
            }
        }
        __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    float* out = partial + (((size_t)blockIdx.y * gmax + g) * chunks + c) * stride;
    if (sh.slices > 1) {
        // slice sums through shared memory (the staging buffers are free),
        // added in slice order by slice 0
        float* red = wsm;
        if (active && slice > 0) {
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y) red[((slice - 1) * sh.tp + t) * 64 + x * 8 + y] = acc[x][y];
        }
        __syncthreads();
        if (active && slice == 0) {
            for (int q = 1; q < sh.slices; ++q)
#pragma unroll
                for (int x = 0; x < 8; ++x)
#pragma unroll
                    for (int y = 0; y < 8; ++y) acc[x][y] += red[((q - 1) * sh.tp + t) * 64 + x * 8 + y];
        }
    }
    if (active && slice == 0) {
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int i = x < 4 ? 4 * ti + x : hm + 4 * ti + x - 4;
            if (i >= mt) continue;
#pragma unroll
            for (int y = 0; y < 8; ++y) {
                const int j = y < 4 ? 4 * tj + y : hn + 4 * tj + y - 4;
                if (j < nt) out[(size_t)(m0 + i) * jb.n + (n0 + j)] = acc[x][y];
            }
        }
    }
    if (bias_col) out[(size_t)jb.m * jb.n + n0 + threadIdx.x] = bsum;
}

size_t wgrad_smem() {
    // two staging buffers; the slice sums reuse them (slices 1.. of at most NTH threads, 64 floats each)
    const size_t stages = sizeof(float) * 2 * WG_STAGE;
    const size_t red = sizeof(float) * (size_t)NTH * 64;
    return stages > red ? stages : red;
}

__global__ void wgrad_reduce_kernel(WgJobs jobs, int n_jobs, int chunks, size_t stride, int gmax,
                                    const float* __restrict__ partial, float* __restrict__ grad) {
    for (int q = 0; q < n_jobs; ++q) {
        const WgJob jb = jobs.job[q];
        const int groups = jb.groups > 0 ? jb.groups : 1;
        const long long total = (long long)jb.m * jb.n + jb.n;
        for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total * groups;
             idx += (long long)gridDim.x * blockDim.x) {
            const int g = (int)(idx / total);
            const long long k = idx % total;
            float s = 0.0f;
            for (int c = 0; c < chunks; ++c) s += partial[(((size_t)q * gmax + g) * chunks + c) * stride + k];
            float* dst = grad + (size_t)g * jb.w_gstride;
            if (k < (long long)jb.m * jb.n) dst[jb.w_off + k] = s;
            else if (jb.b_off >= 0) dst[jb.b_off + (k - (long long)jb.m * jb.n)] = s;
        }
    }
}

// Transposes of `count` row-major [rows][cols] matrices, src + q * src_stride
// to dst + q * rows * cols.
__global__ void transpose_batched_kernel(const float* __restrict__ src, size_t src_stride, int rows, int cols,
                                         int count, float* __restrict__ dst) {
    const size_t per = (size_t)rows * cols;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < per * count;
         k += (size_t)gridDim.x * blockDim.x) {
        const size_t q = k / per, e = k % per;
        const int r = (int)(e / cols), c = (int)(e % cols);
        dst[q * per + (size_t)c * rows + r] = src[q * src_stride + e];
    }
}

// Per-agent advantage moments of a grouped minibatch (one CTA per agent,
// fixed-order tree reduction), and their totals into the minibatch sums.
__global__ void agent_moments_kernel(MbDesc d, int agents, const float* __restrict__ adv, double* moments,
                                     double* stats) {
    __shared__ double ss[2][NTH];
    const int agent = blockIdx.x;
    double s = 0.0, q = 0.0;
    mb_rows_strided(d, threadIdx.x, NTH, [&](int, uint32_t r) {
        const double v = adv[(size_t)r * agents + agent];
        s += v;
        q += v * v;
    });
    ss[0][threadIdx.x] = s;
    ss[1][threadIdx.x] = q;
    __syncthreads();
    for (int o = NTH / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[0][threadIdx.x] += ss[0][threadIdx.x + o];
            ss[1][threadIdx.x] += ss[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        moments[2 * agent] = ss[0][0];
        moments[2 * agent + 1] = ss[1][0];
        atomicAdd(&stats[ST_ADV_SUM], ss[0][0]);
        atomicAdd(&stats[ST_ADV_SQ], ss[1][0]);
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.0f - b1) * gk;
        const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

}  // namespace

size_t fwd_bwd_smem(int in_pad, int H, int O) {
    const int ldo = ((O + 3) & ~3) + 4;
    return sizeof(float) * ((size_t)PTILE * in_pad + 3 * (size_t)PTILE * (H + 4) + (size_t)PTILE * ldo + 2 * PTILE);
}

ej_status launch_gae(const float* rew, const float* value, const uint8_t* done, int T, int rows,
                     int per_env, float gamma, float lam, float* adv, float* ret, cudaStream_t s) {
    int grid = (rows + 255) / 256;
    if (grid > device_sms() * 8) grid = device_sms() * 8;
    gae_kernel<<<grid, 256, 0, s>>>(rew, value, done, T, rows, per_env, gamma, lam, adv, ret);
    return cudaGetLastError() == cudaSuccess ? EJ_OK : fail(EJ_ERR_CUDA, "gae launch failed");
}

ej_status launch_adv_stats(const MbDesc& mb, const float* adv, double* stats, cudaStream_t s) {
    zero_kernel<<<1, 32, 0, s>>>(stats, ST_COUNT_);
    int grid = (mb.count + 255) / 256;
    if (grid > device_sms() * 4) grid = device_sms() * 4;
    if (grid < 1) grid = 1;
    adv_stats_kernel<<<grid, 256, 0, s>>>(mb, adv, stats);
    return cudaGetLastError() == cudaSuccess ? EJ_OK : fail(EJ_ERR_CUDA, "advantage statistics launch failed");
}

ej_status launch_mb_rows_stats(const MbDesc& mb, const float* adv, uint32_t* rows, double* stats, cudaStream_t s) {
    zero_kernel<<<1, 32, 0, s>>>(stats, ST_COUNT_);
    int grid = (mb.count + 255) / 256;
    if (grid > device_sms() * 8) grid = device_sms() * 8;
    if (grid < 1) grid = 1;
    mb_rows_stats_kernel<<<grid, 256, 0, s>>>(mb, adv, rows, stats);
    return cudaGetLastError() == cudaSuccess ? EJ_OK : fail(EJ_ERR_CUDA, "minibatch rows launch failed");
}

ej_status launch_minibatch_grad(const FbArgs& fa, const WgJobs& jobs, int n_jobs, float* partial,
                                size_t stride, int chunks, const float* w2, const float* w3, const float* v2,
                                float* grad, cudaStream_t s) {
    if (fwd_bwd_smem(fa.in_pad, fa.H, fa.O) > 227u * 1024u)
        return fail(EJ_ERR_UNSUPPORTED, "float32 PPO: %d inputs, hidden %d and %d logits need %zu bytes of shared memory "
                    "per 32-row tile (at most %u)", fa.in_dim, fa.H, fa.O, fwd_bwd_smem(fa.in_pad, fa.H, fa.O), 227u * 1024u);
    // transposed copies of the weights the backward pass multiplies by (per agent)
    const int na = fa.agents ? fa.agents : 1, nc = fa.agents && fa.critic_stride ? fa.agents : 1;
    transpose_batched_kernel<<<64 * na, 256, 0, s>>>(w3, fa.actor_stride, fa.H, fa.O, na, fa.w3t);
    transpose_batched_kernel<<<64 * na, 256, 0, s>>>(w2, fa.actor_stride, fa.H, fa.H, na, fa.w2t);
    transpose_batched_kernel<<<64 * nc, 256, 0, s>>>(v2, fa.critic_stride, fa.H, fa.H, nc, fa.v2t);
    zero_kernel<<<1, 32, 0, s>>>(fa.stats, ST_COUNT_);
    if (fa.agents) {
        agent_moments_kernel<<<fa.agents, NTH, 0, s>>>(fa.mb, fa.agents, fa.adv, const_cast<double*>(fa.agent_moments),
                                                      fa.stats);
    } else {
        int grid = (fa.mb.count + 255) / 256;
        if (grid > device_sms() * 4) grid = device_sms() * 4;
        adv_stats_kernel<<<grid, 256, 0, s>>>(fa.mb, fa.adv, fa.stats);
    }
    const size_t smem = fwd_bwd_smem(fa.in_pad, fa.H, fa.O);
    static SmemOptIn opt_in;
    ej_status st = opt_in.ensure((const void*)fwd_bwd_kernel, smem);
    if (st != EJ_OK) return st;
    const int n_tiles = na * ((fa.mb.count + PTILE - 1) / PTILE);
    // as many CTAs as fit an SM (three at hidden 128, two at 256)
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fwd_bwd_kernel, NTH, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int g2 = n_tiles < per_sm * device_sms() ? n_tiles : per_sm * device_sms();
    fwd_bwd_kernel<<<g2, NTH, smem, s>>>(fa);
    int zt = 1, gmax = 1;
    for (int q = 0; q < n_jobs; ++q) {
        const int g = jobs.job[q].groups > 0 ? jobs.job[q].groups : 1;
        const int t = g * ((jobs.job[q].m + WG_TILE - 1) / WG_TILE) * ((jobs.job[q].n + WG_TILE - 1) / WG_TILE);
        zt = t > zt ? t : zt;
        gmax = g > gmax ? g : gmax;
    }
    static SmemOptIn wg_opt_in;
    if ((st = wg_opt_in.ensure((const void*)wgrad_kernel, wgrad_smem())) != EJ_OK) return st;
    wgrad_kernel<<<dim3(chunks, n_jobs, zt), NTH, wgrad_smem(), s>>>(jobs, na * fa.mb.count, chunks, stride, gmax,
                                                                     partial);
    wgrad_reduce_kernel<<<device_sms() * 4, 256, 0, s>>>(jobs, n_jobs, chunks, stride, gmax, partial, grad);
    return cudaGetLastError() == cudaSuccess ? EJ_OK : fail(EJ_ERR_CUDA, "minibatch gradient launch failed");
}

namespace {
__global__ void minibatch_loss_kernel(double* stats, int count, const double* moments, float vf_coef, float ent_coef) {
    if (threadIdx.x == 0) {
        const double n = moments ? moments[0] : (double)count;
        const double sum = stats[ST_PG] + (double)vf_coef * stats[ST_VF] - (double)ent_coef * stats[ST_ENT];
        stats[ST_LOSS] = n > 0.0 ? sum / n : 0.0;
    }
}
}  // namespace

ej_status launch_minibatch_loss(double* stats, int count, const double* moments, float vf_coef, float ent_coef,
                                cudaStream_t s) {
    minibatch_loss_kernel<<<1, 32, 0, s>>>(stats, count, moments, vf_coef, ent_coef);
    return cudaGetLastError() == cudaSuccess ? EJ_OK : fail(EJ_ERR_CUDA, "minibatch loss launch failed");
}

ej_status launch_adam(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                      float eps, int step, cudaStream_t s) {
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    int grid = (int)((n + 255) / 256);
    if (grid > device_sms() * 4) grid = device_sms() * 4;
    adam_kernel<<<grid, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? EJ_OK : fail(EJ_ERR_CUDA, "adam launch failed");
}

}  // namespace ej
