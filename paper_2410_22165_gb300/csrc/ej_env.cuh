// EconoJax environment step on sm_103a (arxiv 2410.22165, Section 3): the
// kernel template.  ej_env.cu instantiates it for any resource / price-level
// count (read from the parameters at run time); ej_env_r2p5.cu for the
// default market of Table 2 (2 resources, 5 price levels), ej_env_r2p10.cu and
// ej_env_r2p20.cu for the finer price grids, with those counts known at
// compile time, so that every per-level loop unrolls and every division by the
// number of levels becomes a multiply.
//
// One CTA runs one environment; thread i is population agent i.  The CTA
// loads the environment's state from HBM once, runs n_steps steps with the
// agents' scalars in registers and their per-resource arrays, the order book
// and all per-step scratch in shared memory, and stores the state once.
// Per step, HBM sees only the streamed inputs (actions, draws) and the
// outputs (rewards, observations, masks).
//
// Order book: per environment, per (resource, side, price level) a FIFO of
// 4-byte orders (placed step << 16 | agent), packed level after level in
// shared memory.  Within a level the FIFO is in priority order (older first;
// orders of one step sorted by their random key), so matching and expiry
// only ever remove a prefix of each level and a step's new orders append.
#pragma once

#include <cfloat>
#include <cmath>

#include "ej_internal.cuh"

namespace ej {
namespace envk {

constexpr unsigned FULL = 0xFFFFFFFFu;

// Resource and price-level counts: compile-time when RC / PC > 0.
template <int RC> __device__ __forceinline__ int nR(const KParams& p) { return RC > 0 ? RC : p.R; }
template <int PC> __device__ __forceinline__ int nP(const KParams& p) { return PC > 0 ? PC : p.P; }
template <int RC, int PC> __device__ __forceinline__ int nW(const KParams& p) {
    return (RC > 0 && PC > 0) ? (2 + RC + 2 * RC * PC + 31) / 32 : p.W;
}

struct Sm {
    int* inv;    // [R][NT] liquid units
    int* inve;   // [R][NT] units in escrow
    float* sg;   // [R][NT] gather skill
    uint32_t* book;            // [cap] resting orders, level after level
    uint32_t* book_alt;        // [cap] the compacted book of this step is written here, then swapped
    int* lvl_old;              // [L]   resting orders per level
    int* lvl_start;            // [L+1] their start in book
    int* lvl_new;              // [L]   orders placed this step per level
    int* lvl_nstart;           // [L+1]
    int* lvl_n;                // [L]   old + new
    int* lvl_rm;               // [L]   removed by matching or expiry
    int* lvl_exp;              // [L]   survivors
    int* lvl_xstart;           // [L+1]
    int* lvl_cstart;           // [L+1] start of survivors in the compacted book
    int* kmatch;               // [R]   trades per resource this step
    int* bid_before;           // [R][P] bids at levels above p
    int* ask_before;           // [R][P] asks at levels below p
    float* rates;              // [EJ_MAX_NB]
    float* mkt;                // [R][4] best bid, best ask, #bids/A_e, #asks/A_e
    float* red;                // [NW][M+1] per-warp partial sums
    float* fin;                // [M+1]
    float* gstat;              // [M][3] mean, std, median
    float* misc;               // [16] gini, prod, share, ugprev, period left, time fraction
    float* nord_frac;          // [max_orders + 1] n / max_orders, rounded once
    // phase A
    unsigned long long* newkey;  // [NT] (tie-break key << 32) | agent, bucketed by level
    uint32_t* newsorted;         // [NT] new orders in priority order, bucketed by level
    int* d_coin; int* d_esc; int* d_inc; int* d_nord;   // [NT] market changes in ticks / counts
    int* d_inv; int* d_inve;                            // [R][NT]
    float* tax;                                         // [NT]
    // phase B / C (alias phase A)
    float* stat;                 // [M][NT]
    float* obs;                  // [NT][D]
};

enum { MISC_GINI = 0, MISC_PROD = 1, MISC_SHARE = 2, MISC_UGPREV = 3, MISC_PLEFT = 4, MISC_TFRAC = 5,
       MISC_PIVOT = 8 };   // MISC_PIVOT + m: key of metric m's last lower middle value (as float bits)

template <int NT>
__device__ __forceinline__ Sm carve(unsigned char* base, const KParams& p) {
    const SmemLayout s = smem_layout(NT, p.R, p.P, p.L, p.cap, p.M, p.D);
    Sm m;
    m.inv = (int*)(base + s.inv);
    m.inve = (int*)(base + s.inve);
    m.sg = (float*)(base + s.sg);
    m.book = (uint32_t*)(base + s.book);
    m.book_alt = (uint32_t*)(base + s.book) + p.cap;
    int* lv = (int*)(base + s.lvl);
    const int L = p.L;
    m.lvl_old = lv;            lv += L;
    m.lvl_start = lv;          lv += L + 1;
    m.lvl_new = lv;            lv += L;
    m.lvl_nstart = lv;         lv += L + 1;
    m.lvl_n = lv;              lv += L;
    m.lvl_rm = lv;             lv += L;
    m.lvl_exp = lv;            lv += L;
    m.lvl_xstart = lv;         lv += L + 1;
    m.lvl_cstart = lv;
    int* kb = (int*)(base + s.kb);
    m.kmatch = kb;             kb += p.R;
    m.bid_before = kb;         kb += p.R * p.P;
    m.ask_before = kb;
    float* fl = (float*)(base + s.fl);
    constexpr int NW = NT / 32;
    m.rates = fl;              fl += EJ_MAX_NB;
    m.mkt = fl;                fl += 4 * p.R;
    m.red = fl;                fl += NW * (p.M + 1);
    m.fin = fl;                fl += p.M + 1;
    m.gstat = fl;              fl += 3 * p.M;
    m.misc = fl;               fl += 16;
    m.nord_frac = fl;
    unsigned char* a = base + s.alias;
    m.newkey = (unsigned long long*)a;  a += align16(8u * NT);
    m.newsorted = (uint32_t*)a;         a += align16(4u * NT);
    m.d_coin = (int*)a;                 a += align16(4u * NT);
    m.d_esc = (int*)a;                  a += align16(4u * NT);
    m.d_inc = (int*)a;                  a += align16(4u * NT);
    m.d_nord = (int*)a;                 a += align16(4u * NT);
    m.d_inv = (int*)a;                  a += align16(4u * p.R * NT);
    m.d_inve = (int*)a;                 a += align16(4u * p.R * NT);
    m.tax = (float*)a;
    m.stat = (float*)(base + s.stat);
    m.obs = (float*)(base + s.alias);
    return m;
}

// Exclusive prefix sum of in[0..n) into out[0..n] (out[n] = total), by one warp.
__device__ __forceinline__ void warp_excl_scan(const int* in, int* out, int n, int lane) {
    int carry = 0;
    for (int base = 0; base < n; base += 32) {
        const int v = (base + lane < n) ? in[base + lane] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (base + lane < n) out[base + lane] = carry + x - v;
        carry += __shfl_sync(FULL, x, 31);
    }
    if (lane == 0) out[n] = carry;
}

// k-th order of level l this step: resting orders first, then this step's.
__device__ __forceinline__ uint32_t seq_get(const Sm& s, int l, int k) {
    const int old = s.lvl_old[l];
    return k < old ? s.book[s.lvl_start[l] + k] : s.newsorted[s.lvl_nstart[l] + k - old];
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ float labor_of(const KParams& p, int ng, int nc, int nt) {
    return __fadd_rn(__fadd_rn(__fmul_rn(p.lg, (float)ng), __fmul_rn(p.lc, (float)nc)),
                     __fmul_rn(p.lt, (float)nt));
}

// Eq. 1, in float.  C^(1-eta) by the hardware exp2 / log2 (__powf: relative
// error about 2e-6 for coin up to 1e5, inside the 1e-5 utility tolerance;
// no integer state depends on it).  4 % of the step at E = 1024 x A = 100.
__device__ __forceinline__ float utility(const KParams& p, float coin, float labor) {
    return __fsub_rn(__fdiv_rn(__fsub_rn(__powf(coin, p.ome), 1.0f), p.ome), labor);
}

// Section 3 "Setting tax rates": marginal tax bracket by bracket, each
// operation rounded once, brackets in ascending order.
__device__ __forceinline__ float bracket_tax(const KParams& p, const float* rates, float income) {
    float tax = 0.0f;
    for (int b = 0; b < p.nb; ++b) {
        const float lo = b == 0 ? 0.0f : p.th[b - 1];
        float part = __fsub_rn(income, lo);
        if (part < 0.0f) part = 0.0f;
        if (b < p.nb - 1) {
            const float width = __fsub_rn(p.th[b], lo);
            if (part > width) part = width;
        }
        tax = __fadd_rn(tax, __fmul_rn(rates[b], part));
    }
    return tax;
}

// Per-agent registers.
struct Agent {
    float coin, income, uprev, sc;
    int esc, nord, ng, nc, nt;
};

template <int NT, int RC>
__device__ __forceinline__ bool craftable(const KParams& p, const Sm& s, int i) {
    const int R = nR<RC>(p);
    int enough = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) enough += s.inv[r * NT + i] >= p.Rk;
    return enough >= p.Rd;
}

// Section 3 "Action masking".
// Skill improvement after a gather or a craft (Section 5): relative gain
// skill_gain shrinking linearly to 0 at skill_max, every operation rounded
// once: s + s * (gain * (1 - s / max)), capped at max.
__device__ __forceinline__ float skill_up(const KParams& p, float sk) {
    const float room = __fsub_rn(1.0f, __fdiv_rn(sk, p.skill_max));
    const float up = __fadd_rn(sk, __fmul_rn(sk, __fmul_rn(p.skill_gain, room)));
    return fminf(up, p.skill_max);
}

template <int NT, int RC, int PC>
__device__ __forceinline__ bool action_valid(const KParams& p, const Sm& s, const Agent& g, int i, int a) {
    const int R = nR<RC>(p), P = nP<PC>(p);
    if (a < 0 || a >= 2 + R + 2 * R * P) return false;
    if (a == 0) return p.allow_noop != 0;
    if (a <= R) return true;
    if (a == R + 1) return craftable<NT, RC>(p, s, i);
    int j = a - (R + 2);
    const int RP = R * P;
    if (j < RP) return g.nord < p.max_orders && g.coin >= p.price[j % P];
    j -= RP;
    return g.nord < p.max_orders && s.inv[(j / P) * NT + i] >= 1;
}

__device__ __forceinline__ void or_bits(uint32_t& word, int w, int pos, uint64_t bits) {
    const int sh = pos - 32 * w;
    if (sh >= 32 || sh <= -64) return;
    const uint64_t v = sh >= 0 ? (bits << sh) : (bits >> (-sh));
    word |= (uint32_t)v;
}

// New episode for agent i (Section 3: skills drawn at initialization; Table 2
// starting coin).
template <int NT, int RC>
__device__ void start_agent(const KParams& p, const Sm& s, Agent& g, int i, int e, uint32_t ep,
                            uint32_t k0, uint32_t k1, bool live) {
    const int R = nR<RC>(p);
    g.coin = live ? p.start_coin : 0.0f;
    g.income = 0.0f;
    g.esc = g.nord = g.ng = g.nc = g.nt = 0;
    g.sc = 0.0f;
    for (int r = 0; r < R; ++r) {
        s.inv[r * NT + i] = 0;
        s.inve[r * NT + i] = 0;
        s.sg[r * NT + i] = 0.0f;
    }
    if (live) {
        if (p.skill_init == 0) {
            // U[0, 1): the uniforms of consecutive chunks give SG[0..R-1], then SC
            const int n_chunks = (R + 1 + 3) / 4;
            for (int c = 0; c < n_chunks; ++c) {
                const uint4 x = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)e, ep, 2u | ((uint32_t)c << 8)), k0, k1);
                const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int idx = 4 * c + j;
                    if (idx < R) s.sg[idx * NT + i] = u01(xs[j]);
                    else if (idx == R) g.sc = u01(xs[j]);
                }
            }
        } else {
            // around 1 with standard deviation 1 (Section 5): 12 uniforms (chunks 3j..3j+2)
            // summed in order, minus 5, clamped to [0, skill_max]; skill j < R gathers r = j
            for (int j = 0; j <= R; ++j) {
                float sum = 0.0f;
                for (int c = 0; c < 3; ++c) {
                    const uint4 x = philox4x32_10(
                        make_uint4((uint32_t)i, (uint32_t)e, ep, 2u | ((uint32_t)(3 * j + c) << 8)), k0, k1);
                    sum = __fadd_rn(sum, u01(x.x));
                    sum = __fadd_rn(sum, u01(x.y));
                    sum = __fadd_rn(sum, u01(x.z));
                    sum = __fadd_rn(sum, u01(x.w));
                }
                const float v = fminf(fmaxf(__fsub_rn(sum, 5.0f), 0.0f), p.skill_max);
                if (j < R) s.sg[j * NT + i] = v;
                else g.sc = v;
            }
        }
        g.uprev = utility(p, g.coin, 0.0f);
    } else {
        g.uprev = 0.0f;
    }
}

// Each agent's values of the government's statistics metrics (total coin,
// period earnings, labor) into s.stat[m][i]; absent agents get +FLT_MAX so
// that they sort last.
template <int NT>
__device__ __forceinline__ void fill_stats(const KParams& p, const Sm& s, const Agent& g, int i, int Ae) {
    if (i < Ae) {
        s.stat[0 * NT + i] = __fadd_rn(g.coin, __fmul_rn(p.tick, (float)g.esc));
        s.stat[1 * NT + i] = g.income;
        s.stat[2 * NT + i] = labor_of(p, g.ng, g.nc, g.nt);
    } else {
        s.stat[0 * NT + i] = FLT_MAX;
        s.stat[1 * NT + i] = FLT_MAX;
        s.stat[2 * NT + i] = FLT_MAX;
    }
}

// Bitonic sort (ascending) of 32*V values held V per lane in lane order:
// element index lane * V + v.  Stages whose partner is in the same lane
// (distance < V) compare registers; the others exchange by shuffles.  The
// direction of a stage depends on the lane only once k >= V.
template <int V>
__device__ __forceinline__ void warp_bitonic(float (&x)[V], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * V; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < V) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if ((v & j) == 0) {
                        const int w = v | j;
                        const bool asc = k < V ? ((v & k) == 0) : ((lane & (k / V)) == 0);
                        const float lo = fminf(x[v], x[w]), hi = fmaxf(x[v], x[w]);
                        x[v] = asc ? lo : hi;
                        x[w] = asc ? hi : lo;
                    }
                }
            } else {
                const int d = j / V;
                const bool asc = (lane & (k / V)) == 0;
                const bool keep_min = ((lane & d) == 0) == asc;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float y = __shfl_xor_sync(FULL, x[v], d);
                    x[v] = keep_min ? fminf(x[v], y) : fmaxf(x[v], y);
                }
            }
        }
    }
}

template <int V>
__device__ __forceinline__ float sorted_at(const float (&x)[V], int k) {
    float v = x[0];
#pragma unroll
    for (int r = 1; r < V; ++r) if ((k % V) == r) v = x[r];
    return __shfl_sync(FULL, v, k / V);
}

// Order-preserving unsigned key of a float (not NaN): a < b <=> key(a) < key(b).
__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// The k-th smallest (from 0) of the 32 V values of a warp (V per lane), found
// by walking from `pivot` (a value near the answer) over the distinct values
// in between: warp-wide counts and minima / maxima per step (redux.sync).
// Exact; false when the walk would take more than `max_steps` steps.
template <int V>
__device__ __forceinline__ bool walk_select(const uint32_t (&key)[V], int k, uint32_t pivot, int max_steps,
                                            uint32_t& out) {
    int lt = 0, le = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) { lt += key[v] < pivot; le += key[v] <= pivot; }
    lt = __reduce_add_sync(FULL, lt);
    le = __reduce_add_sync(FULL, le);
    if (k >= lt && k < le) { out = pivot; return true; }
    uint32_t cur = pivot;
    if (k >= le) {                       // upwards: rank = elements <= cur
        int rank = le;
        for (int it = 0; it < max_steps; ++it) {
            uint32_t mn = 0xFFFFFFFFu;
#pragma unroll
            for (int v = 0; v < V; ++v) mn = key[v] > cur ? min(mn, key[v]) : mn;
            const uint32_t nxt = __reduce_min_sync(FULL, mn);
            int eq = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) eq += key[v] == nxt;
            eq = __reduce_add_sync(FULL, eq);
            if (k < rank + eq) { out = nxt; return true; }
            rank += eq;
            cur = nxt;
        }
    } else {                             // downwards: rank = elements < cur
        int rank = lt;
        for (int it = 0; it < max_steps; ++it) {
            uint32_t mx = 0u;
#pragma unroll
            for (int v = 0; v < V; ++v) mx = key[v] < cur ? max(mx, key[v]) : mx;
            const uint32_t prv = __reduce_max_sync(FULL, mx);
            int eq = 0;
#pragma unroll
            for (int v = 0; v < V; ++v) eq += key[v] == prv;
            rank -= __reduce_add_sync(FULL, eq);
            if (k >= rank) { out = prv; return true; }
            cur = prv;
        }
    }
    return false;
}

// Statistics of one metric by one warp (mean, population std, median; and
// for total coin the gini index and the total, Eq. 5-6), from s.stat[m].
// Total coin is sorted (the gini index weights each value by its rank); the
// other metrics' medians are the two middle order statistics, walked to from
// the previous step's lower middle value (the medians move little from step
// to step), with the sort as the fallback of a long walk.  Same values either
// way.
template <int V>
__device__ void warp_metric_stats(const Sm& s, int m, int lane, int Ae, int NT) {
    constexpr int MAX_WALK = 12;
    float x[V];
    float sum = 0.0f;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int idx = lane * V + v;
        x[v] = s.stat[m * NT + idx];
        if (idx < Ae) sum += x[v];
    }
    sum = warp_sum(sum);
    const float mean = sum / (float)Ae;
    const int k_lo = (Ae - 1) >> 1, k_hi = Ae >> 1;
    float ss = 0.0f, gnum = 0.0f, lo = 0.0f, hi = 0.0f;
    bool walked = false;
    if (m != 0) {
        // values in index order (the sum of squares does not need them sorted)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (lane * V + v < Ae) {
                const float d = x[v] - mean;
                ss += d * d;
            }
        }
        uint32_t key[V];
#pragma unroll
        for (int v = 0; v < V; ++v) key[v] = fkey(x[v]);
        uint32_t klo, khi;
        const uint32_t pivot = __float_as_uint(s.misc[MISC_PIVOT + m]);
        walked = walk_select<V>(key, k_lo, pivot, MAX_WALK, klo) &&
                 walk_select<V>(key, k_hi, klo, MAX_WALK, khi);
        if (walked) {
            lo = fkey_inv(klo);
            hi = fkey_inv(khi);
            __syncwarp();
            if (lane == 0) s.misc[MISC_PIVOT + m] = __uint_as_float(klo);
        }
    }
    if (!walked) {
        warp_bitonic<V>(x, lane);
        ss = 0.0f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int idx = lane * V + v;
            if (idx < Ae) {
                const float d = x[v] - mean;
                ss += d * d;
                gnum += (float)(2 * idx - Ae + 1) * x[v];
            }
        }
        lo = sorted_at<V>(x, k_lo);
        hi = sorted_at<V>(x, k_hi);
        if (m != 0 && lane == 0) s.misc[MISC_PIVOT + m] = __uint_as_float(fkey(lo));
    }
    ss = warp_sum(ss);
    if (m == 0) gnum = warp_sum(gnum);
    if (lane == 0) {
        s.gstat[3 * m + 0] = mean;
        s.gstat[3 * m + 1] = sqrtf(ss / (float)Ae);
        s.gstat[3 * m + 2] = (Ae & 1) ? hi : 0.5f * (lo + hi);
        if (m == 0) {
            s.misc[MISC_PROD] = sum;
            s.misc[MISC_GINI] = sum > 0.0f ? gnum / ((float)Ae * sum) : 0.0f;
        }
    }
}

// Block-wide bitonic sort of M arrays of NT floats (ascending), for CTAs
// too wide for the register sort.
template <int NT>
__device__ void block_bitonic(float* a, int M) {
    const int i = threadIdx.x;
#pragma unroll 1
    for (int k = 2; k <= NT; k <<= 1) {
#pragma unroll 1
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int ixj = i ^ j;
            if (ixj > i) {
                const bool asc = (i & k) == 0;
                for (int m = 0; m < M; ++m) {
                    const float x = a[m * NT + i], y = a[m * NT + ixj];
                    if ((x > y) == asc) { a[m * NT + i] = y; a[m * NT + ixj] = x; }
                }
            }
            __syncthreads();
        }
    }
}

// Population statistics (Sec. 3; App. A: the government sees mean, std and
// median) from s.stat, which fill_stats wrote before a barrier.  Results in
// s.gstat and s.misc, for readers after the next barrier (CTAs of up to 128
// threads sort one metric per warp with no barrier, so the sorting warps can
// run into the next step's first phase while the others start it).
template <int NT>
__device__ void population_stats(const KParams& p, const Sm& s, int i, int Ae) {
    constexpr int NW = NT / 32;
    const int lane = i & 31, warp = i >> 5;
    const int M = p.M;
    if constexpr (NT <= 128) {
        constexpr int V = NT / 32;
        for (int m = warp; m < M; m += NW) warp_metric_stats<V>(s, m, lane, Ae, NT);
    } else {
        block_bitonic<NT>(s.stat, M);
        for (int m = warp; m < M; m += NW) {
            // sums over the sorted array by one warp
            float sum = 0.0f, gnum = 0.0f;
            for (int idx = lane; idx < Ae; idx += 32) {
                const float v = s.stat[m * NT + idx];
                sum += v;
                gnum += (float)(2 * idx - Ae + 1) * v;
            }
            sum = warp_sum(sum);
            gnum = warp_sum(gnum);
            const float mean = sum / (float)Ae;
            float ss = 0.0f;
            for (int idx = lane; idx < Ae; idx += 32) {
                const float d = s.stat[m * NT + idx] - mean;
                ss += d * d;
            }
            ss = warp_sum(ss);
            if (lane == 0) {
                const float lo = s.stat[m * NT + ((Ae - 1) >> 1)], hi = s.stat[m * NT + (Ae >> 1)];
                s.gstat[3 * m + 0] = mean;
                s.gstat[3 * m + 1] = sqrtf(ss / (float)Ae);
                s.gstat[3 * m + 2] = (Ae & 1) ? hi : 0.5f * (lo + hi);
                if (m == 0) {
                    s.misc[MISC_PROD] = sum;
                    s.misc[MISC_GINI] = sum > 0.0f ? gnum / ((float)Ae * sum) : 0.0f;
                }
            }
        }
    }
}

__device__ __forceinline__ float social_welfare(const KParams& p, const Sm& s) {
    // Eq. 3-5 (READING of the garbled Eq. 4: omega (1 - gini) + 1 - omega)
    return (p.omega * (1.0f - s.misc[MISC_GINI]) + (1.0f - p.omega)) * s.misc[MISC_PROD];
}

// Market statistics of the resting book for the observation (App. A:
// highest bid, lowest ask, number of orders), from per-level counts.
template <int RC, int PC>
__device__ __forceinline__ void market_stats(const KParams& p, const Sm& s, const int* counts, int i, int Ae) {
    const int R = nR<RC>(p), P = nP<PC>(p);
    if (i < R) {
        const int lb = (i * 2) * P, la = (i * 2 + 1) * P;
        int hi = -1, lo = P, nbids = 0, nasks = 0;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int cb = counts[lb + q], ca = counts[la + q];
            nbids += cb;
            nasks += ca;
            if (cb > 0) hi = q;
            if (ca > 0 && lo == P) lo = q;
        }
        s.mkt[4 * i + 0] = hi >= 0 ? p.price[hi] : 0.0f;
        s.mkt[4 * i + 1] = lo < P ? p.price[lo] : 0.0f;
        s.mkt[4 * i + 2] = __fdiv_rn((float)nbids, (float)Ae);
        s.mkt[4 * i + 3] = __fdiv_rn((float)nasks, (float)Ae);
    }
}

// Per-step uniform values of the observation (fraction of the tax period
// left, fraction of the episode elapsed), by one thread into s.misc.
__device__ __forceinline__ void time_features(const KParams& p, const Sm& s, int t) {
    s.misc[MISC_PLEFT] = __fdiv_rn((float)(p.T_tax - t % p.T_tax), (float)p.T_tax);
    s.misc[MISC_TFRAC] = __fdiv_rn((float)t, (float)p.T_ep);
}

// Government observation of output row `row` (thread i writes entry i):
// statistics, rates, time features.
__device__ __forceinline__ void write_gobs(const KParams& p, const Sm& s, const DevIO& io, size_t row, int i) {
    if (io.gobs && i < p.G) {
        const int nst = 3 * p.M;
        float v;
        if (i < nst) v = s.gstat[i];
        else if (i < nst + p.nb) v = s.rates[i - nst];
        else if (i == nst + p.nb) v = s.misc[MISC_PLEFT];
        else v = s.misc[MISC_TFRAC];
        io.gobs[row * p.G + i] = v;
    }
}

// Population observations and action masks of the current state for output
// row `row` (each warp stages and writes its own agents' rows; no barrier at
// the end: every warp has finished reading its staging slots when it leaves,
// except in CTAs of 256 and more threads, whose two staging rounds end with
// a barrier each).
template <int NT, int RC, int PC>
__device__ void observe_rows(const KParams& p, const Sm& s, const Agent& g, const DevIO& io, size_t row, int i,
                             int Ae) {
    const int R = nR<RC>(p), P = nP<PC>(p), D = p.D, W = nW<RC, PC>(p);
    const int lane = i & 31, warp = i >> 5;
    const float period_left = s.misc[MISC_PLEFT];
    const float time_frac = s.misc[MISC_TFRAC];
    if (io.mask && i < p.A) {
        const bool live = i < Ae;
        const bool room = g.nord < p.max_orders;
        if (W == 1) {
            // every action bit fits one word: build it directly
            uint32_t word = 0;
            if (live) {
                uint32_t buy_bits = 0;
                if (room) {
#pragma unroll
                    for (int q = 0; q < P; ++q) buy_bits |= (uint32_t)(g.coin >= p.price[q]) << q;
                }
                const uint32_t all_p = (1u << P) - 1u;
                word = (p.allow_noop ? 1u : 0u) | (((1u << R) - 1u) << 1);
                if (craftable<NT, RC>(p, s, i)) word |= 1u << (R + 1);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    word |= buy_bits << (R + 2 + r * P);
                    if (room && s.inv[r * NT + i] >= 1) word |= all_p << (R + 2 + R * P + r * P);
                }
            }
            io.mask[row * p.A + i] = word;
        } else {
            uint64_t buy_bits = 0;
            if (room)
                for (int q = 0; q < P; ++q) buy_bits |= (uint64_t)(g.coin >= p.price[q]) << q;
            const uint64_t all_p = (1ull << P) - 1;
            const bool craft = craftable<NT, RC>(p, s, i);
            for (int w = 0; w < W; ++w) {
                uint32_t word = 0;
                if (live) {
                    if (p.allow_noop) or_bits(word, w, 0, 1);
                    or_bits(word, w, 1, (1ull << R) - 1);
                    if (craft) or_bits(word, w, R + 1, 1);
                    for (int r = 0; r < R; ++r) {
                        or_bits(word, w, R + 2 + r * P, buy_bits);
                        if (room && s.inv[r * NT + i] >= 1) or_bits(word, w, R + 2 + R * P + r * P, all_p);
                    }
                }
                io.mask[(row * p.A + i) * W + w] = word;
            }
        }
    }
    // observations: each warp stages its 32 rows in shared memory and copies
    // them out with 16-byte stores; in CTAs of 256 and 512 threads half of the
    // warps at a time share the staging slots (two rounds), which halves the
    // buffer so that 4 and 2 such CTAs fit an SM
    constexpr int NW = NT / 32, ROUNDS = NT >= 256 ? 2 : 1, HALF = NW / ROUNDS;
    for (int round = 0; round < ROUNDS; ++round) {
    if (io.obs && warp / HALF == round) {
        const int first = warp * 32;
        if (first < p.A) {
            if (i < p.A) {
                float* o = s.obs + (size_t)(i - round * HALF * 32) * D;
                if (i < Ae) {
                    int k = 0;
                    o[k++] = g.coin;
                    o[k++] = __fmul_rn(p.tick, (float)g.esc);
                    o[k++] = labor_of(p, g.ng, g.nc, g.nt);
#pragma unroll
                    for (int r = 0; r < R; ++r) o[k + r] = (float)s.inv[r * NT + i];
                    k += R;
#pragma unroll
                    for (int r = 0; r < R; ++r) o[k + r] = (float)s.inve[r * NT + i];
                    k += R;
#pragma unroll
                    for (int r = 0; r < R; ++r) o[k + r] = s.sg[r * NT + i];
                    k += R;
                    o[k++] = g.sc;
                    o[k++] = s.nord_frac[g.nord];
#pragma unroll
                    for (int q = 0; q < 4 * R; ++q) o[k + q] = s.mkt[q];
                    k += 4 * R;
                    for (int b = 0; b < p.nb; ++b) o[k + b] = s.rates[b];
                    k += p.nb;
                    o[k++] = g.income;
                    o[k++] = period_left;
                    o[k++] = time_frac;
                } else {
                    for (int k = 0; k < D; ++k) o[k] = 0.0f;
                }
            }
            __syncwarp();
            const int rows = min(32, p.A - first);
            const int n = rows * D;
            const float* src = s.obs + (size_t)(first - round * HALF * 32) * D;
            float* dst = io.obs + (row * p.A + first) * (size_t)D;
            if ((n & 3) == 0 && (((uintptr_t)dst) & 15) == 0) {
                const float4* src4 = (const float4*)src;
                float4* dst4 = (float4*)dst;
                for (int j = lane; j < (n >> 2); j += 32) dst4[j] = src4[j];
            } else {
                for (int j = lane; j < n; j += 32) dst[j] = src[j];
            }
        }
    }
    if (ROUNDS > 1) __syncthreads();
    }
}

// Observation, government observation and action mask of the current state
// (Sec. 3; App. A), written for output row `row`.  Needs s.mkt, s.gstat,
// s.rates and the time features in s.misc.  Ends with a barrier.
template <int NT, int RC, int PC>
__device__ void observe(const KParams& p, const Sm& s, const Agent& g, const DevIO& io, size_t row, int i,
                        int Ae) {
    write_gobs(p, s, io, row, i);
    observe_rows<NT, RC, PC>(p, s, g, io, row, i, Ae);
    __syncthreads();
}

// CTAs per SM each instantiation must fit (registers: 72 per thread at 7
// CTAs of 128 threads, 64 at 4 of 256 and 2 of 512, none spilled; the shared
// memory of 100-, 250- and 500-agent environments fits the same counts), so
// that a batch of environments runs in as few waves as possible: e.g. 1024
// environments of 100 agents in one wave of 7 x 152 CTAs.  (8 CTAs of 128
// threads fit at 64 registers, but were slower: 12.2 against 10.6 ms per
// 1000-step episode of 1024 x 100.)
template <int NT> struct MinCtas { static constexpr int value = NT <= 32 ? 16 : NT <= 64 ? 12 : NT <= 128 ? 7 : NT <= 256 ? 4 : 2; };

template <int NT, int RC, int PC>
__global__ void __launch_bounds__(NT, MinCtas<NT>::value) env_kernel(KParams p, DevState st, DevIO io, int n_steps,
                                                                     int mode, uint32_t seed_lo, uint32_t seed_hi) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm s = carve<NT>(smem_raw, p);
    const int e = p.e0 + (int)blockIdx.x;
    const int i = threadIdx.x;
    const int lane = i & 31, warp = i >> 5;
    constexpr int NW = NT / 32;
    const int R = nR<RC>(p), P = nP<PC>(p), L = 2 * R * P;
    const size_t ea = (size_t)e * p.A_s;
    const int owner = NT - 1 - i;          // levels l = owner, owner + NT, ... belong to this thread

    if (i <= p.max_orders) s.nord_frac[i] = __fdiv_rn((float)i, (float)(p.max_orders > 0 ? p.max_orders : 1));
    if (i < 3) s.misc[MISC_PIVOT + i] = __uint_as_float(fkey(0.0f));   // any start works: the walk is exact
    Agent g;
    int t;
    uint32_t gs, ep, k0, k1;
    int Ae;
    if (mode & MODE_RESET) {
        Ae = io.pop_sizes ? io.pop_sizes[e] : p.A;
        Ae = Ae < 1 ? 1 : (Ae > p.A ? p.A : Ae);
        k0 = seed_lo;
        k1 = seed_hi;
        t = 0; gs = 0; ep = 0;
        start_agent<NT, RC>(p, s, g, i, e, 0u, k0, k1, i < Ae);
        for (int l = i; l < L; l += NT) s.lvl_old[l] = 0;
        for (int l = i; l <= L; l += NT) s.lvl_start[l] = 0;
        if (i < EJ_MAX_NB) s.rates[i] = 0.0f;
        if (e == 0 && i == 0) { st.key[0] = k0; st.key[1] = k1; }
        if (i == 0) time_features(p, s, t);
        fill_stats<NT>(p, s, g, i, Ae);
        __syncthreads();
        market_stats<RC, PC>(p, s, s.lvl_old, i, Ae);
        population_stats<NT>(p, s, i, Ae);
        __syncthreads();
        if (i == 0) s.misc[MISC_UGPREV] = social_welfare(p, s);
        observe<NT, RC, PC>(p, s, g, io, (size_t)e, i, Ae);
    } else {
        Ae = st.pop[e];
        k0 = st.key[0];
        k1 = st.key[1];
        t = st.t[e]; gs = st.gstep[e]; ep = st.episode[e];
        if (i < p.A_s) {
            g.coin = st.coin[ea + i]; g.esc = st.esc[ea + i]; g.income = st.income[ea + i];
            g.uprev = st.uprev[ea + i]; g.nord = st.nord[ea + i]; g.sc = st.sc[ea + i];
            const size_t c3 = (size_t)e * 3 * p.A_s;
            g.ng = st.counts[c3 + i]; g.nc = st.counts[c3 + p.A_s + i]; g.nt = st.counts[c3 + 2 * p.A_s + i];
            for (int r = 0; r < R; ++r) {
                const size_t k = ((size_t)e * R + r) * p.A_s + i;
                s.inv[r * NT + i] = st.inv[k]; s.inve[r * NT + i] = st.inve[k]; s.sg[r * NT + i] = st.sg[k];
            }
        } else {
            g.coin = g.income = g.uprev = g.sc = 0.0f;
            g.esc = g.nord = g.ng = g.nc = g.nt = 0;
            for (int r = 0; r < R; ++r) { s.inv[r * NT + i] = 0; s.inve[r * NT + i] = 0; s.sg[r * NT + i] = 0.0f; }
        }
        for (int l = i; l < L; l += NT) s.lvl_old[l] = st.lvl[(size_t)e * L + l];
        if (i < EJ_MAX_NB) s.rates[i] = st.rates[(size_t)e * EJ_MAX_NB + i];
        if (i == 0) s.misc[MISC_UGPREV] = st.ugprev[e];
        __syncthreads();
        if (warp == 0) warp_excl_scan(s.lvl_old, s.lvl_start, L, lane);
        __syncthreads();
        const int nbook = s.lvl_start[L];
        for (int j = i; j < nbook; j += NT) s.book[j] = st.book[(size_t)e * p.cap + j];
    }
    // per-step scratch starts at zero (later steps clear it after use)
    for (int l = i; l < L; l += NT) s.lvl_new[l] = 0;
    __syncthreads();

    // Per step, six barriers: (1) after the own action, (2) after the new
    // orders' keys, (3) after their ranking, (4) after matching and expiry,
    // (5) after the survivors' compaction and the market deltas, (6) after
    // the rewards, statistics inputs and observations.  The 20-level prefix
    // sums are computed by every warp in registers (no barrier of their own),
    // and the statistics sorts of step k run after barrier (6) without a
    // barrier behind them: their results (the government reward and
    // observation of row k) are written in step k+1's second phase, or after
    // the loop for the last step.
    const bool reg_scan = L <= 32;
    bool pending = false;                     // government outputs of the previous row not yet written
    size_t prev_row = 0;
    for (int step = 0; step < n_steps; ++step) {
        const size_t row = (size_t)step * p.E + e;
        const bool live = i < Ae;
        // ---- inputs of this step
        int a = 0;
        float gu = 0.0f;
        uint32_t tbk = 0;
        if (live) {
            if (mode & (MODE_POP_DRAW | MODE_AUX_DRAW)) {
                const uint4 x = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)e, gs, 0u), k0, k1);
                a = below(x.x, p.nA);
                gu = u01(x.y);
                tbk = x.z;
            }
            if (!(mode & MODE_POP_DRAW)) a = io.act[row * p.A + i];
            if (!(mode & MODE_AUX_DRAW)) {
                const size_t k = row * p.A + i;
                gu = io.gather_u[k];
                tbk = io.tb[k];
            }
        }
        // this agent's market deltas start at zero (only this thread touched them before the barrier)
        s.d_coin[i] = 0; s.d_esc[i] = 0; s.d_inc[i] = 0; s.d_nord[i] = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) { s.d_inv[r * NT + i] = 0; s.d_inve[r * NT + i] = 0; }

        // 1. the agent's own action (Sec. 3 "Population Agents")
        int my_l = -1, my_slot = 0;
        if (live && a != 0 && action_valid<NT, RC, PC>(p, s, g, i, a)) {
            if (a <= R) {                                   // gather resource a-1
                const int r = a - 1;
                const float rho = __fmul_rn(p.gather_rho, gu);
                const float sum = __fadd_rn(s.sg[r * NT + i], rho);
                s.inv[r * NT + i] += (int)floorf(sum);
                g.ng += 1;
                if (p.skill_gain > 0.0f) s.sg[r * NT + i] = skill_up(p, s.sg[r * NT + i]);
            } else if (a == R + 1) {                        // craft
                uint32_t used = 0;
                for (int k = 0; k < p.Rd; ++k) {
                    int best = -1, bv = 0;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int v = s.inv[r * NT + i];
                        if (!((used >> r) & 1u) && (best < 0 || v > bv)) { best = r; bv = v; }
                    }
                    used |= 1u << best;
                    s.inv[best * NT + i] = bv - p.Rk;
                }
                const float gain = __fmul_rn(g.sc, p.craft_coin);
                g.coin = __fadd_rn(g.coin, gain);
                g.income = __fadd_rn(g.income, gain);
                g.nc += 1;
                if (p.skill_gain > 0.0f) g.sc = skill_up(p, g.sc);
            } else {                                        // one order into escrow
                int j = a - (R + 2);
                const int side = j >= R * P;
                if (side) j -= R * P;
                const int r = j / P, q = j % P;
                if (side == 0) {
                    g.coin = __fsub_rn(g.coin, p.price[q]);
                    g.esc += p.ticks[q];
                } else {
                    s.inv[r * NT + i] -= 1;
                    s.inve[r * NT + i] += 1;
                }
                g.nord += 1;
                g.nt += 1;
                my_l = (r * 2 + side) * P + q;
                my_slot = atomicAdd(&s.lvl_new[my_l], 1);
            }
        }
        __syncthreads();                                                        // (1)

        // the previous row's government reward and observation (its statistics
        // were sorted after the previous step's last barrier); the rate
        // entries are written by the threads that own the rates, before 0.
        if (pending) {
            if (i == 0) {
                const float ug = social_welfare(p, s);
                if (io.grew) io.grew[prev_row] = __fsub_rn(ug, s.misc[MISC_UGPREV]);
                s.misc[MISC_UGPREV] = ug;
            }
            if (io.gobs && i < p.G && (i < 3 * p.M || i >= 3 * p.M + p.nb)) write_gobs(p, s, io, prev_row, i);
        }
        if (pending && io.gobs && i < p.nb) io.gobs[prev_row * p.G + 3 * p.M + i] = s.rates[i];
        // 0. period start: the government's rate levels take effect (read by
        //    the tax and the observations after later barriers)
        if (p.gov_enabled && t % p.T_tax == 0 && i < p.nb) {
            int lev;
            if (mode & MODE_GOV_DRAW) {
                const uint4 x = philox4x32_10(make_uint4(0u, (uint32_t)e, gs, 1u), k0, k1);
                lev = below(i == 0 ? x.x : i == 1 ? x.y : i == 2 ? x.z : x.w, p.tax_levels);
            } else {
                lev = io.gov_act[row * p.nb + i];
            }
            lev = lev < 0 ? 0 : (lev > p.tax_levels - 1 ? p.tax_levels - 1 : lev);
            s.rates[i] = __fdiv_rn((float)lev, (float)(p.tax_levels - 1));
        }

        // where this step's orders go; trades per resource K = max_q min(#bids >= q, #asks <= q)
        if (reg_scan) {
            // every warp scans the 20-odd level counts in registers
            const int v = lane < L ? s.lvl_new[lane] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += y;
            }
            const int excl = x - v;
            if (warp == 0) {
                if (lane < L) s.lvl_nstart[lane] = excl;
                if (lane == 31) s.lvl_nstart[L] = x;
            }
            const int start = __shfl_sync(FULL, excl, my_l < 0 ? 0 : my_l);
            if (my_l >= 0) s.newkey[start + my_slot] = ((unsigned long long)tbk << 32) | (uint32_t)i;
        } else if (warp == 0) {
            warp_excl_scan(s.lvl_new, s.lvl_nstart, L, lane);
        }
        for (int r = warp; r < R; r += NW) {
            const int q = lane;
            const int lb = (r * 2) * P + q, la = (r * 2 + 1) * P + q;
            const int bc = q < P ? s.lvl_old[lb] + s.lvl_new[lb] : 0;
            const int ac = q < P ? s.lvl_old[la] + s.lvl_new[la] : 0;
            int B = bc, S = ac;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int vb = __shfl_down_sync(FULL, B, o);
                if (lane + o < 32) B += vb;
                const int va = __shfl_up_sync(FULL, S, o);
                if (lane >= o) S += va;
            }
            int m = q < P ? min(B, S) : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
            if (q < P) {
                s.bid_before[r * P + q] = B - bc;
                s.ask_before[r * P + q] = S - ac;
                s.lvl_n[lb] = bc;
                s.lvl_n[la] = ac;
            }
            if (lane == 0) s.kmatch[r] = m;
        }
        if (!reg_scan) {
            __syncthreads();
            if (my_l >= 0) s.newkey[s.lvl_nstart[my_l] + my_slot] = ((unsigned long long)tbk << 32) | (uint32_t)i;
        }
        __syncthreads();                                                        // (2)
        // this step's orders in priority order within their level (random key, then agent)
        if (my_l >= 0) {
            const unsigned long long mk = ((unsigned long long)tbk << 32) | (uint32_t)i;
            const int st0 = s.lvl_nstart[my_l], cnt = s.lvl_new[my_l];
            int rank = 0;
            for (int j = 0; j < cnt; ++j) rank += s.newkey[st0 + j] < mk;
            s.newsorted[st0 + rank] = ((uint32_t)t << 16) | (uint32_t)i;
        }
        __syncthreads();                                                        // (3)

        // 2. matching (Sec. 3 "Trading"; App. A): pair k = k-th best bid with k-th
        //    best ask; resource r's trades start on warp r (mod the CTA)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int K = s.kmatch[r];
            const int base = (r * 32) % NT;
            for (int k = (i - base + NT) % NT; k < K; k += NT) {
                int qb = P - 1;
                while (k >= s.bid_before[r * P + qb] + s.lvl_n[(r * 2) * P + qb]) --qb;
                int qa = 0;
                while (k >= s.ask_before[r * P + qa] + s.lvl_n[(r * 2 + 1) * P + qa]) ++qa;
                const uint32_t ob = seq_get(s, (r * 2) * P + qb, k - s.bid_before[r * P + qb]);
                const uint32_t oa = seq_get(s, (r * 2 + 1) * P + qa, k - s.ask_before[r * P + qa]);
                const int buyer = ob & 0xFFFF, seller = oa & 0xFFFF;
                const int tk_bid = p.ticks[qb];
                const int tk = (ob >> 16) > (oa >> 16) ? tk_bid : p.ticks[qa];   // price of the later order
                atomicAdd(&s.d_esc[buyer], tk_bid);
                atomicAdd(&s.d_coin[buyer], tk_bid - tk);
                atomicAdd(&s.d_inv[r * NT + buyer], 1);
                atomicAdd(&s.d_nord[buyer], 1);
                atomicAdd(&s.d_inve[r * NT + seller], 1);
                atomicAdd(&s.d_coin[seller], tk);
                atomicAdd(&s.d_inc[seller], tk);
                atomicAdd(&s.d_nord[seller], 1);
            }
        }
        // 3. expiry (level owners): after the matched prefix, the orders that have
        //    now taken part in `expire` rounds leave; escrow goes back
        const int thr = t + 1 - p.expire;
        for (int l = owner; l < L; l += NT) {
            const int r = l / (2 * P), side = (l / P) & 1, q = l % P;
            const int n = s.lvl_n[l];
            const int before = side ? s.ask_before[r * P + q] : s.bid_before[r * P + q];
            int idx = s.kmatch[r] - before;
            idx = idx < 0 ? 0 : (idx > n ? n : idx);
            while (idx < n) {
                const uint32_t o = seq_get(s, l, idx);
                if ((int)(o >> 16) > thr) break;
                const int who = o & 0xFFFF;
                if (side == 0) {
                    atomicAdd(&s.d_coin[who], p.ticks[q]);
                    atomicAdd(&s.d_esc[who], p.ticks[q]);
                } else {
                    atomicAdd(&s.d_inv[r * NT + who], 1);
                    atomicAdd(&s.d_inve[r * NT + who], 1);
                }
                atomicAdd(&s.d_nord[who], 1);
                ++idx;
            }
            s.lvl_rm[l] = idx;                  // removed by matching or expiry
            s.lvl_exp[l] = n - idx;             // survivors
        }
        __syncthreads();                                                        // (4)
        // survivors into the other book buffer, one warp per level, at their
        // compacted start (every warp scans the survivor counts in registers)
        int cx = 0;
        if (reg_scan) {
            const int v = lane < L ? s.lvl_exp[lane] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += y;
            }
            cx = x - v;
            if (warp == 0) {
                if (lane < L) s.lvl_cstart[lane] = cx;
                if (lane == 31) s.lvl_cstart[L] = x;
            }
        } else {
            if (warp == 0) warp_excl_scan(s.lvl_exp, s.lvl_cstart, L, lane);
            __syncthreads();
        }
        for (int l = warp; l < L; l += NW) {
            const int c = s.lvl_exp[l], src0 = s.lvl_rm[l];
            const int dst0 = reg_scan ? __shfl_sync(FULL, cx, l) : s.lvl_cstart[l];
            const int old = s.lvl_old[l], ostart = s.lvl_start[l], nstart = s.lvl_nstart[l];
            for (int j = lane; j < c; j += 32) {
                const int k = src0 + j;
                s.book_alt[dst0 + j] = k < old ? s.book[ostart + k] : s.newsorted[nstart + k - old];
            }
        }
        market_stats<RC, PC>(p, s, s.lvl_exp, i, Ae);
        if (live) {
            g.coin = __fadd_rn(g.coin, __fmul_rn(p.tick, (float)s.d_coin[i]));
            g.income = __fadd_rn(g.income, __fmul_rn(p.tick, (float)s.d_inc[i]));
            g.esc -= s.d_esc[i];
            g.nord -= s.d_nord[i];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                s.inv[r * NT + i] += s.d_inv[r * NT + i];
                s.inve[r * NT + i] -= s.d_inve[r * NT + i];
            }
        }
        if (i == 0) time_features(p, s, (t + 1) == p.T_ep ? 0 : t + 1);
        __syncthreads();                                                        // (5)
        { uint32_t* tmp = s.book; s.book = s.book_alt; s.book_alt = tmp; }
        for (int l = owner; l < L; l += NT) {
            s.lvl_old[l] = s.lvl_exp[l];
            s.lvl_start[l] = s.lvl_cstart[l];
            s.lvl_new[l] = 0;               // the next step's tickets (read last before the compaction)
        }
        if (owner == 0) s.lvl_start[L] = s.lvl_cstart[L];

        // 4. period end: bracket tax, equal redistribution, new period of earnings
        if ((t + 1) % p.T_tax == 0) {
            if (p.gov_enabled) {
                float tax = 0.0f;
                if (live) {
                    tax = bracket_tax(p, s.rates, g.income);
                    if (tax > g.coin) tax = g.coin;
                }
                // pool: each block of 32 agents summed as a butterfly (offsets
                // 16, 8, 4, 2, 1), the blocks then added in agent order
                float v = tax;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(FULL, v, o));
                if (lane == 0) s.red[warp] = v;
                __syncthreads();
                float pool = 0.0f;
                for (int w = 0; w < NW; ++w) pool = __fadd_rn(pool, s.red[w]);
                if (live) g.coin = __fadd_rn(__fsub_rn(g.coin, tax), __fdiv_rn(pool, (float)Ae));
            }
            g.income = 0.0f;
        }

        // 5. rewards: Eq. 2 on Eq. 1 (the government's follows from the statistics)
        if (live) {
            const float c = __fadd_rn(g.coin, __fmul_rn(p.tick, (float)g.esc));
            const float u = utility(p, c, labor_of(p, g.ng, g.nc, g.nt));
            if (io.rew) io.rew[row * p.A + i] = __fsub_rn(u, g.uprev);
            g.uprev = u;
        } else if (io.rew && i < p.A) {
            io.rew[row * p.A + i] = 0.0f;
        }
        fill_stats<NT>(p, s, g, i, Ae);

        // 6. end of episode: functional reset with the next episode's skills
        t += 1;
        gs += 1;
        const bool ended = t == p.T_ep;
        if (io.done && i == 0) io.done[row] = ended ? 1 : 0;
        // 7. observation of the new state (at an episode end: of the next episode's first state, below)
        if (!ended) observe_rows<NT, RC, PC>(p, s, g, io, row, i, Ae);
        __syncthreads();                                                        // (6)
        population_stats<NT>(p, s, i, Ae);
        pending = true;
        prev_row = row;
        if (ended) {
            __syncthreads();
            if (i == 0) {
                const float ug = social_welfare(p, s);
                if (io.grew) io.grew[row] = __fsub_rn(ug, s.misc[MISC_UGPREV]);
            }
            t = 0;
            ep += 1;
            __syncthreads();
            start_agent<NT, RC>(p, s, g, i, e, ep, k0, k1, live);
            for (int l = i; l < L; l += NT) s.lvl_old[l] = 0;
            for (int l = i; l <= L; l += NT) s.lvl_start[l] = 0;
            if (i < EJ_MAX_NB) s.rates[i] = 0.0f;
            fill_stats<NT>(p, s, g, i, Ae);
            __syncthreads();
            market_stats<RC, PC>(p, s, s.lvl_old, i, Ae);
            population_stats<NT>(p, s, i, Ae);
            __syncthreads();
            if (i == 0) s.misc[MISC_UGPREV] = social_welfare(p, s);
            observe_rows<NT, RC, PC>(p, s, g, io, row, i, Ae);
            __syncthreads();
            // the reset state's statistics stand for this row's government observation;
            // its reward is written
            if (io.gobs && i < p.G) write_gobs(p, s, io, row, i);
            pending = false;
        }
    }
    if (pending) {
        __syncthreads();
        if (i == 0) {
            const float ug = social_welfare(p, s);
            if (io.grew) io.grew[prev_row] = __fsub_rn(ug, s.misc[MISC_UGPREV]);
            s.misc[MISC_UGPREV] = ug;
        }
        write_gobs(p, s, io, prev_row, i);
    }
    __syncthreads();

    // ---- store the state
    if (i < p.A_s) {
        st.coin[ea + i] = g.coin; st.esc[ea + i] = g.esc; st.income[ea + i] = g.income;
        st.uprev[ea + i] = g.uprev; st.nord[ea + i] = g.nord; st.sc[ea + i] = g.sc;
        const size_t c3 = (size_t)e * 3 * p.A_s;
        st.counts[c3 + i] = g.ng; st.counts[c3 + p.A_s + i] = g.nc; st.counts[c3 + 2 * p.A_s + i] = g.nt;
        for (int r = 0; r < R; ++r) {
            const size_t k = ((size_t)e * R + r) * p.A_s + i;
            st.inv[k] = s.inv[r * NT + i]; st.inve[k] = s.inve[r * NT + i]; st.sg[k] = s.sg[r * NT + i];
        }
    }
    for (int l = i; l < L; l += NT) st.lvl[(size_t)e * L + l] = s.lvl_old[l];
    const int nbook = s.lvl_start[L];
    for (int j = i; j < nbook; j += NT) st.book[(size_t)e * p.cap + j] = s.book[j];
    if (i < EJ_MAX_NB) st.rates[(size_t)e * EJ_MAX_NB + i] = s.rates[i];
    if (i == 0) {
        st.t[e] = t; st.gstep[e] = gs; st.episode[e] = ep; st.pop[e] = Ae;
        st.ugprev[e] = s.misc[MISC_UGPREV];
    }
}

// Launch of one instantiation with its dynamic shared memory.
template <int NT, int RC, int PC>
ej_status launch_nt(const KParams& kp, const Layout& lay, const DevState& st, const DevIO& io,
                    int n_steps, int mode, uint64_t seed, cudaStream_t stream) {
    const int smem = lay.sizes.smem_bytes;
    static SmemOptIn opt_in;     // per instantiation, per device
    ej_status st_opt = opt_in.ensure((const void*)env_kernel<NT, RC, PC>, (size_t)smem);
    if (st_opt != EJ_OK) return st_opt;
    env_kernel<NT, RC, PC><<<kp.ne, NT, smem, stream>>>(kp, st, io, n_steps, mode, (uint32_t)seed,
                                                        (uint32_t)(seed >> 32));
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "env kernel launch: %s", cudaGetErrorString(err));
    return EJ_OK;
}

}  // namespace envk
}  // namespace ej
