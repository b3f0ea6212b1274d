// C ABI of the PPO update: parameters, workspace sizing, advantages,
// minibatch gradients, Adam, and the whole update.
#include <cmath>
#include <cstring>

#include "ej_internal.cuh"
#include "ej_ppo.cuh"

namespace ej {

namespace {

constexpr int WG_CHUNKS = 96;   // row chunks of the split-K weight-gradient kernel
constexpr int WG_CHUNKS_AGENT = 8;   // row chunks per agent of per-agent networks' gradients

struct NetDims { int in, O, heads, head, rows_per_step; };

NetDims dims(const KParams& kp, int net) {
    NetDims d;
    if (net == EJ_NET_POP) { d.in = kp.D; d.heads = 1; d.head = kp.nA; d.rows_per_step = kp.E * kp.A; }
    else { d.in = kp.G; d.heads = kp.nb; d.head = kp.tax_levels; d.rows_per_step = kp.E; }
    d.O = d.heads * d.head;
    return d;
}

uint64_t a256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// Workspace regions (byte offsets).
struct Ws {
    uint64_t adv[2], ret[2], stats[2], totals, wt3, wt2, wv2, rows, partial, grad[2], total;
    uint64_t row_floats;   // floats of the per-row buffers (largest minibatch of either network)
    uint64_t max_mb;       // rows of the largest minibatch
    uint64_t wg_stride;    // floats of one weight-gradient job's partial sums
    uint64_t amom;         // per-agent advantage moments (per-agent networks)
};

// agents > 0: the population's networks are per agent (room for A sets of
// transposed weights, per-agent moments, partial sums per agent and an A-fold
// population gradient).  The advantages and returns sit at the same offsets
// for every value of agents.
Ws ws_layout(const KParams& kp, const EjPpoParams* pp, int T, int H, int agents = 0) {
    Ws w;
    uint64_t o = 0;
    const uint64_t na = agents > 0 ? (uint64_t)agents : 1;
    const NetDims dp = dims(kp, EJ_NET_POP), dg = dims(kp, EJ_NET_GOV);
    const NetDims dd[2] = {dp, dg};
    for (int n = 0; n < 2; ++n) {
        const uint64_t N = (uint64_t)T * dd[n].rows_per_step;
        w.adv[n] = o; o = a256(o + 4 * N);
        w.ret[n] = o; o = a256(o + 4 * N);
    }
    w.stats[0] = o; o = a256(o + 8 * ST_COUNT_);
    w.stats[1] = o; o = a256(o + 8 * ST_COUNT_);
    w.totals = o; o = a256(o + 8 * 2 * ST_COUNT_);
    const int Omax = dp.O > dg.O ? dp.O : dg.O;
    w.wt3 = o; o = a256(o + 4ull * Omax * H * na);
    w.wt2 = o; o = a256(o + 4ull * H * H * na);
    w.wv2 = o; o = a256(o + 4ull * H * H * na);
    w.amom = o; o = a256(o + 8ull * 2 * na);
    uint64_t region = 0, mb = 0;
    for (int n = 0; n < 2; ++n) {
        const uint64_t f = dd[n].in + 8ull * H + dd[n].O + 1;   // x, h1, h2, g1, g2, dl, dz2, dz1, dy2, dy1, dv
        const uint64_t N = (uint64_t)T * dd[n].rows_per_step;
        const uint64_t m = (N + pp->minibatches - 1) / pp->minibatches;
        if (f * m > region) region = f * m;
        if (m > mb) mb = m;
    }
    if (agents > 0) {
        // every agent takes ceil(T E / M) positions of a minibatch
        const uint64_t m = na * (((uint64_t)T * kp.E + pp->minibatches - 1) / pp->minibatches);
        const uint64_t f = dp.in + 8ull * H + dp.O + 1;
        if (f * m > region) region = f * m;
        if (m > mb) mb = m;
    }
    w.row_floats = region;
    w.max_mb = mb;
    w.rows = o; o = a256(o + 4ull * region);
    size_t stride = 0;
    for (int n = 0; n < 2; ++n) {
        const size_t s = wg_stride(dd[n].in, H, dd[n].O);
        stride = s > stride ? s : stride;
    }
    w.wg_stride = stride;
    const uint64_t chunk_sets = agents > 0 && WG_CHUNKS_AGENT * na > WG_CHUNKS ? WG_CHUNKS_AGENT * na : WG_CHUNKS;
    w.partial = o; o = a256(o + 4ull * 6 * chunk_sets * stride);
    for (int n = 0; n < 2; ++n) {
        w.grad[n] = o;
        o = a256(o + 4ull * net_offsets(dd[n].in, H, dd[n].O).total * (n == 0 ? na : 1));
    }
    w.total = o;
    return w;
}

int domain_bits(uint64_t N) {
    int b = 2;
    while ((1ull << b) < N) ++b;
    return b;
}

ej_status check_common(const EjParams* p, const EjPpoParams* pp, int T, int H, Layout* lay, KParams* kp) {
    ej_status st = derive(p, lay, kp);
    if (st != EJ_OK) return st;
    if (!pp) return fail(EJ_ERR_ARG, "ppo params is NULL");
    if (T < 1) return fail(EJ_ERR_ARG, "T must be >= 1");
    if (pp->minibatches < 1 || pp->epochs < 1) return fail(EJ_ERR_ARG, "epochs and minibatches must be >= 1");
    // every minibatch of every network holds at least one row (the government
    // network has the fewest: T x E)
    if ((uint64_t)pp->minibatches > (uint64_t)T * (uint64_t)kp->E)
        return fail(EJ_ERR_ARG, "%d minibatches exceed the government network's %llu rows (T x E)", pp->minibatches,
                    (unsigned long long)T * (unsigned long long)kp->E);
    if (H < 32 || H > 256 || H % 32) return fail(EJ_ERR_UNSUPPORTED, "PPO update supports hidden 32 .. 256 in steps of 32");
    if (kp->nb * p->tax_levels > 128 || kp->nA > 128 || kp->D > 128 || kp->G > 128)
        return fail(EJ_ERR_UNSUPPORTED, "PPO update needs inputs and logits <= 128");
    if ((uint64_t)T * kp->E * kp->A >= (1ull << 31)) return fail(EJ_ERR_UNSUPPORTED, "too many rows");
    return EJ_OK;
}

}  // namespace

// The gradient kernels take network `net` (-1: both) at this precision: the
// float32 32-row tile fits shared memory; the BF16 kernel's fixed widths hold
// the shape.  Checked before anything is launched.
ej_status check_grad_shape(const KParams& kp, int H, int precision, int net) {
    for (int n = 0; n < 2; ++n) {
        if (net >= 0 && n != net) continue;
        const int in = n == EJ_NET_POP ? kp.D : kp.G;
        const int O = n == EJ_NET_POP ? kp.nA : kp.nb * kp.tax_levels;
        if (precision == EJ_BF16) {
            const ej_status st = bf16_grad_shape(in, H, O, n == EJ_NET_POP ? 1 : kp.nb, n == EJ_NET_POP ? kp.W : 0);
            if (st != EJ_OK) return st;
            continue;
        }
        const size_t smem = fwd_bwd_smem((in + 3) & ~3, H, O);
        if (smem > 227u * 1024u)
            return fail(EJ_ERR_UNSUPPORTED, "float32 PPO: %d inputs, hidden %d and %d logits need %zu bytes of shared "
                        "memory per 32-row tile (at most %u)", in, H, O, smem, 227u * 1024u);
    }
    return EJ_OK;
}

// Every rollout-buffer array a PPO call reads is present: for GAE (`gae`)
// the rewards, values and done flags, for a minibatch gradient the inputs,
// mask, actions, old log-probabilities and values of the network (net =
// EJ_NET_POP, EJ_NET_GOV, or -1 for both).
ej_status check_rollout(const EjRollout* b, int net, bool gae, bool grad) {
    if (!b) return fail(EJ_ERR_ARG, "rollout buffer is NULL");
    const bool pop = net != EJ_NET_GOV, gov = net != EJ_NET_POP;
    struct { const void* p; bool need; const char* name; } f[] = {
        {b->rew, gae && pop, "rew"}, {b->value, (gae || grad) && pop, "value"}, {b->done, gae, "done"},
        {b->grew, gae && gov, "grew"}, {b->gvalue, (gae || grad) && gov, "gvalue"},
        {b->obs, grad && pop, "obs"}, {b->mask, grad && pop, "mask"}, {b->act, grad && pop, "act"},
        {b->logp, grad && pop, "logp"}, {b->gobs, grad && gov, "gobs"}, {b->gact, grad && gov, "gact"},
        {b->glogp, grad && gov, "glogp"},
    };
    for (const auto& x : f)
        if (x.need && !x.p) return fail(EJ_ERR_ARG, "rollout buffer member %s is NULL", x.name);
    return EJ_OK;
}

namespace {

// Minibatch m of the permutation keyed by (seed, ctr) over the T x rows-per-step rows of `net`.
MbDesc mb_desc(const KParams& kp, const EjPpoParams* pp, int T, int net, uint32_t ctr, int m) {
    const NetDims d = dims(kp, net);
    const uint64_t N = (uint64_t)T * d.rows_per_step;
    MbDesc mb;
    mb.lo = (int)((N * m) / pp->minibatches);
    mb.count = (int)((N * (m + 1)) / pp->minibatches) - mb.lo;
    mb.N = (uint32_t)N;
    mb.bits = domain_bits(N);
    mb.k0 = (uint32_t)pp->seed;
    mb.k1 = (uint32_t)(pp->seed >> 32);
    mb.ctr = ctr;
    return mb;
}

// Minibatch m of the permutation of the T x E (step, environment) positions,
// taken for every agent (per-agent networks).
MbDesc mb_desc_positions(const KParams& kp, const EjPpoParams* pp, int T, uint32_t ctr, int m) {
    const uint64_t N = (uint64_t)T * kp.E;
    MbDesc mb;
    mb.lo = (int)((N * m) / pp->minibatches);
    mb.count = (int)((N * (m + 1)) / pp->minibatches) - mb.lo;
    mb.N = (uint32_t)N;
    mb.bits = domain_bits(N);
    mb.k0 = (uint32_t)pp->seed;
    mb.k1 = (uint32_t)(pp->seed >> 32);
    mb.ctr = ctr;
    return mb;
}

__global__ void moments_out_kernel(const double* stats, int count, double* out) {
    if (threadIdx.x == 0) {
        out[0] = (double)count;
        out[1] = stats[ST_ADV_SUM];
        out[2] = stats[ST_ADV_SQ];
    }
}

ej_status minibatch_grad(const KParams& kp, const EjPpoParams* pp, int T, int H, int precision, int net,
                         const float* weights, const EjRollout* b, char* ws, const Ws& W, uint32_t ctr,
                         int m, float* grad, double* stats, cudaStream_t s, const double* moments = nullptr) {
    const NetDims d = dims(kp, net);
    const NetOffsets off = net_offsets(d.in, H, d.O);
    FbArgs fa;
    memset(&fa, 0, sizeof fa);
    fa.mb = mb_desc(kp, pp, T, net, ctr, m);
    fa.moments = moments;
    fa.in_dim = d.in; fa.in_pad = (d.in + 3) & ~3; fa.H = H; fa.O = d.O;
    fa.n_heads = d.heads; fa.head = d.head; fa.W = net == EJ_NET_POP ? kp.W : 0;
    fa.clip = pp->clip; fa.vf_coef = pp->vf_coef; fa.vclip = pp->vclip; fa.ent_coef = pp->ent_coef;
    fa.weights = weights;
    if (net == EJ_NET_POP) {
        fa.x = b->obs; fa.mask = b->mask; fa.act = b->act; fa.logp_old = b->logp; fa.v_old = b->value;
    } else {
        fa.x = b->gobs; fa.mask = nullptr; fa.act = b->gact; fa.logp_old = b->glogp; fa.v_old = b->gvalue;
    }
    fa.adv = (const float*)(ws + W.adv[net]);
    fa.ret = (const float*)(ws + W.ret[net]);
    fa.w3t = (float*)(ws + W.wt3); fa.w2t = (float*)(ws + W.wt2); fa.v2t = (float*)(ws + W.wv2);
    fa.stats = stats;
    ej_status st;
    if (precision == EJ_BF16) {
        fa.rows = (uint32_t*)(ws + W.rows);      // the float32 path's per-row region holds >= count entries
        st = launch_ppo_bf16(fa, (float*)(ws + W.partial), 4ull * 6 * WG_CHUNKS * W.wg_stride, grad, s);
        if (st != EJ_OK) return st;
        return launch_minibatch_loss(stats, fa.mb.count, moments, pp->vf_coef, pp->ent_coef, s);
    }
    const uint64_t R = (uint64_t)fa.mb.count;
    float* rb = (float*)(ws + W.rows);
    // hidden-width arrays first: each starts on a 16-byte boundary (H is a multiple of 32)
    fa.ws_h1 = rb; rb += R * H;
    fa.ws_h2 = rb; rb += R * H;
    fa.ws_g1 = rb; rb += R * H;
    fa.ws_g2 = rb; rb += R * H;
    fa.ws_dz2 = rb; rb += R * H;
    fa.ws_dz1 = rb; rb += R * H;
    fa.ws_dy2 = rb; rb += R * H;
    fa.ws_dy1 = rb; rb += R * H;
    fa.ws_x = rb; rb += R * d.in;
    fa.ws_dl = rb; rb += R * d.O;
    fa.ws_dv = rb;
    WgJobs jobs;
    memset(&jobs, 0, sizeof jobs);
    auto job = [&](int q, const float* A, int m_, const float* B, int n_, size_t wo, size_t bo) {
        jobs.job[q].A = A; jobs.job[q].B = B; jobs.job[q].lda = m_; jobs.job[q].ldb = n_;
        jobs.job[q].m = m_; jobs.job[q].n = n_; jobs.job[q].w_off = (long long)wo; jobs.job[q].b_off = (long long)bo;
    };
    job(0, fa.ws_x, d.in, fa.ws_dz1, H, off.W1, off.b1);
    job(1, fa.ws_h1, H, fa.ws_dz2, H, off.W2, off.b2);
    job(2, fa.ws_h2, H, fa.ws_dl, d.O, off.W3, off.b3);
    job(3, fa.ws_x, d.in, fa.ws_dy1, H, off.V1, off.c1);
    job(4, fa.ws_g1, H, fa.ws_dy2, H, off.V2, off.c2);
    job(5, fa.ws_g2, H, fa.ws_dv, 1, off.V3, off.c3);
    if (cudaMemsetAsync(grad, 0, sizeof(float) * off.total, s) != cudaSuccess)
        return fail(EJ_ERR_CUDA, "memset of the gradient failed");
    st = launch_minibatch_grad(fa, jobs, 6, (float*)(ws + W.partial), W.wg_stride, WG_CHUNKS, weights + off.W2,
                               weights + off.W3, weights + off.V2, grad, s);
    if (st != EJ_OK) return st;
    return launch_minibatch_loss(stats, fa.mb.count, moments, pp->vf_coef, pp->ent_coef, s);
}

// Gradient of one minibatch's loss of the population's per-agent networks
// (float32): agent i's actor on agent i's rows; the critic per agent
// (independent) or shared over all agents' rows (CTDE).
ej_status minibatch_grad_agents(const KParams& kp, const EjPpoParams* pp, int T, int H, int layout,
                                const float* weights, const EjRollout* b, char* ws, const Ws& W, uint32_t ctr,
                                int m, float* grad, double* stats, cudaStream_t s) {
    const NetDims d = dims(kp, EJ_NET_POP);
    const NetOffsets off = net_offsets(d.in, H, d.O);
    const int Ag = kp.A;
    FbArgs fa;
    memset(&fa, 0, sizeof fa);
    fa.mb = mb_desc_positions(kp, pp, T, ctr, m);
    fa.in_dim = d.in; fa.in_pad = (d.in + 3) & ~3; fa.H = H; fa.O = d.O;
    fa.n_heads = d.heads; fa.head = d.head; fa.W = kp.W;
    fa.clip = pp->clip; fa.vf_coef = pp->vf_coef; fa.vclip = pp->vclip; fa.ent_coef = pp->ent_coef;
    fa.weights = weights;
    fa.x = b->obs; fa.mask = b->mask; fa.act = b->act; fa.logp_old = b->logp; fa.v_old = b->value;
    fa.adv = (const float*)(ws + W.adv[EJ_NET_POP]);
    fa.ret = (const float*)(ws + W.ret[EJ_NET_POP]);
    fa.w3t = (float*)(ws + W.wt3); fa.w2t = (float*)(ws + W.wt2); fa.v2t = (float*)(ws + W.wv2);
    fa.stats = stats;
    fa.agents = Ag;
    fa.actor_stride = off.total;
    fa.critic_stride = layout == EJ_NETS_INDEPENDENT ? off.total : 0;
    fa.agent_moments = (const double*)(ws + W.amom);
    const uint64_t cnt = (uint64_t)fa.mb.count, R = (uint64_t)Ag * cnt;
    float* rb = (float*)(ws + W.rows);
    // hidden-width arrays first: each starts on a 16-byte boundary (H is a multiple of 32)
    fa.ws_h1 = rb; rb += R * H;
    fa.ws_h2 = rb; rb += R * H;
    fa.ws_g1 = rb; rb += R * H;
    fa.ws_g2 = rb; rb += R * H;
    fa.ws_dz2 = rb; rb += R * H;
    fa.ws_dz1 = rb; rb += R * H;
    fa.ws_dy2 = rb; rb += R * H;
    fa.ws_dy1 = rb; rb += R * H;
    fa.ws_x = rb; rb += R * d.in;
    fa.ws_dl = rb; rb += R * d.O;
    fa.ws_dv = rb;
    WgJobs jobs;
    memset(&jobs, 0, sizeof jobs);
    auto job = [&](int q, const float* A, int m_, const float* B, int n_, size_t wo, size_t bo, bool per_agent) {
        WgJob& j = jobs.job[q];
        j.A = A; j.B = B; j.lda = m_; j.ldb = n_; j.m = m_; j.n = n_;
        j.w_off = (long long)wo; j.b_off = (long long)bo;
        j.groups = per_agent ? Ag : 1;
        j.group_rows = per_agent ? (int)cnt : (int)R;
        j.w_gstride = per_agent ? (long long)off.total : 0;
    };
    const bool critic_per_agent = layout == EJ_NETS_INDEPENDENT;
    job(0, fa.ws_x, d.in, fa.ws_dz1, H, off.W1, off.b1, true);
    job(1, fa.ws_h1, H, fa.ws_dz2, H, off.W2, off.b2, true);
    job(2, fa.ws_h2, H, fa.ws_dl, d.O, off.W3, off.b3, true);
    job(3, fa.ws_x, d.in, fa.ws_dy1, H, off.V1, off.c1, critic_per_agent);
    job(4, fa.ws_g1, H, fa.ws_dy2, H, off.V2, off.c2, critic_per_agent);
    job(5, fa.ws_g2, H, fa.ws_dv, 1, off.V3, off.c3, critic_per_agent);
    if (cudaMemsetAsync(grad, 0, sizeof(float) * off.total * Ag, s) != cudaSuccess)
        return fail(EJ_ERR_CUDA, "memset of the gradient failed");
    ej_status st = launch_minibatch_grad(fa, jobs, 6, (float*)(ws + W.partial), W.wg_stride, WG_CHUNKS_AGENT,
                                         weights + off.W2, weights + off.W3, weights + off.V2, grad, s);
    if (st != EJ_OK) return st;
    return launch_minibatch_loss(stats, (int)R, nullptr, pp->vf_coef, pp->ent_coef, s);
}

ej_status check_agents(int layout, int precision) {
    if (layout != EJ_NETS_INDEPENDENT && layout != EJ_NETS_CTDE) return fail(EJ_ERR_ARG, "unknown network layout %d", layout);
    if (precision != EJ_FP32) return fail(EJ_ERR_UNSUPPORTED, "per-agent networks run in FP32 (precision %d)", precision);
    return EJ_OK;
}

__global__ void accumulate_stats_kernel(const double* st, double* totals) {
    const int k = threadIdx.x;
    if (k < ST_COUNT_) totals[k] += st[k];
}

__global__ void finalize_stats_kernel(const double* totals, double rows_pop, double rows_gov, float* out) {
    const int k = threadIdx.x;
    if (k < 2 * 5) {
        const int net = k / 5, q = k % 5;
        const double n = net == 0 ? rows_pop : rows_gov;
        out[net * 8 + q] = (float)(totals[net * ST_COUNT_ + ST_PG + q] / n);
    }
}

}  // namespace

}  // namespace ej

using namespace ej;

extern "C" {

ej_status ej_ppo_params_default(EjPpoParams* pp) {
    if (!pp) return fail(EJ_ERR_ARG, "NULL");
    memset(pp, 0, sizeof *pp);
    pp->gamma = 0.99f; pp->lam = 0.95f; pp->clip = 0.2f; pp->vf_coef = 0.25f; pp->vclip = 10.0f;
    pp->ent_coef = 0.1f; pp->lr = 5e-4f; pp->beta1 = 0.9f; pp->beta2 = 0.999f; pp->eps = 1e-5f;
    pp->epochs = 4; pp->minibatches = 8; pp->seed = 0;
    return EJ_OK;
}

ej_status ej_ppo_workspace_bytes(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                                 uint64_t* bytes) {
    Layout lay;
    KParams kp;
    ej_status st = check_common(p, pp, T, hidden, &lay, &kp);
    if (st != EJ_OK) return st;
    if (bytes) *bytes = ws_layout(kp, pp, T, hidden).total;
    return EJ_OK;
}

ej_status ej_ppo_workspace_offsets(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                                   uint64_t* offsets) {
    Layout lay;
    KParams kp;
    ej_status st = check_common(p, pp, T, hidden, &lay, &kp);
    if (st != EJ_OK) return st;
    if (!offsets) return fail(EJ_ERR_ARG, "NULL");
    const Ws W = ws_layout(kp, pp, T, hidden);
    offsets[0] = W.adv[0]; offsets[1] = W.ret[0]; offsets[2] = W.adv[1]; offsets[3] = W.ret[1];
    return EJ_OK;
}

ej_status ppo_advantages(const EjParams* p, const EjPpoParams* pp, int32_t T, const EjRollout* b,
                         void* workspace, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = check_common(p, pp, T, 128, &lay, &kp);
    if (st != EJ_OK) return st;
    if (!b || !workspace) return fail(EJ_ERR_ARG, "NULL rollout or workspace");
    if ((st = check_rollout(b, -1, true, false)) != EJ_OK) return st;
    if ((uintptr_t)workspace % 256) return fail(EJ_ERR_ARG, "workspace must be 256-byte aligned");
    const Ws W = ws_layout(kp, pp, T, 128);
    char* ws = (char*)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    st = launch_gae(b->rew, b->value, b->done, T, kp.E * kp.A, kp.A, pp->gamma, pp->lam,
                    (float*)(ws + W.adv[0]), (float*)(ws + W.ret[0]), s);
    if (st != EJ_OK) return st;
    return launch_gae(b->grew, b->gvalue, b->done, T, kp.E, 1, pp->gamma, pp->lam,
                      (float*)(ws + W.adv[1]), (float*)(ws + W.ret[1]), s);
}

ej_status ppo_minibatch_grad(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                             int32_t precision, int32_t net, const float* weights, const EjRollout* b,
                             void* workspace, uint32_t shuffle_ctr, int32_t minibatch, float* grad,
                             double* stats_out, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = check_common(p, pp, T, hidden, &lay, &kp);
    if (st != EJ_OK) return st;
    if (precision != EJ_FP32 && precision != EJ_BF16) return fail(EJ_ERR_ARG, "unknown precision %d", precision);
    if (net != EJ_NET_POP && net != EJ_NET_GOV) return fail(EJ_ERR_ARG, "unknown network %d", net);
    if (!b || !workspace || !weights || !grad) return fail(EJ_ERR_ARG, "NULL argument");
    if ((st = check_rollout(b, net, false, true)) != EJ_OK) return st;
    if ((st = check_grad_shape(kp, hidden, precision, net)) != EJ_OK) return st;
    if ((uintptr_t)workspace % 256 || (uintptr_t)weights % 16) return fail(EJ_ERR_ARG, "misaligned buffer");
    if (minibatch < 0 || minibatch >= pp->minibatches) return fail(EJ_ERR_ARG, "minibatch out of range");
    const Ws W = ws_layout(kp, pp, T, hidden);
    char* ws = (char*)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    double* stats = (double*)(ws + W.stats[net]);
    st = minibatch_grad(kp, pp, T, hidden, precision, net, weights, b, ws, W, shuffle_ctr, minibatch, grad, stats, s);
    if (st != EJ_OK) return st;
    if (stats_out) {
        if (cudaMemcpyAsync(stats_out, stats, sizeof(double) * ST_COUNT_, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(EJ_ERR_CUDA, "stats copy failed");
    }
    return EJ_OK;
}

ej_status ppo_minibatch_moments(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t net,
                                const EjRollout* b, void* workspace, uint32_t shuffle_ctr, int32_t minibatch,
                                double* moments, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = check_common(p, pp, T, 128, &lay, &kp);
    if (st != EJ_OK) return st;
    if (net != EJ_NET_POP && net != EJ_NET_GOV) return fail(EJ_ERR_ARG, "unknown network %d", net);
    if (!b || !workspace || !moments) return fail(EJ_ERR_ARG, "NULL argument");
    if ((uintptr_t)workspace % 256) return fail(EJ_ERR_ARG, "misaligned workspace");
    if (minibatch < 0 || minibatch >= pp->minibatches) return fail(EJ_ERR_ARG, "minibatch out of range");
    const Ws W = ws_layout(kp, pp, T, 128);
    char* ws = (char*)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    const MbDesc mb = mb_desc(kp, pp, T, net, shuffle_ctr, minibatch);
    double* stats = (double*)(ws + W.stats[net]);
    if ((st = launch_adv_stats(mb, (const float*)(ws + W.adv[net]), stats, s)) != EJ_OK) return st;
    moments_out_kernel<<<1, 32, 0, s>>>(stats, mb.count, moments);
    return cudaGetLastError() == cudaSuccess ? EJ_OK : fail(EJ_ERR_CUDA, "moments launch failed");
}

ej_status ppo_minibatch_grad_global(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                                    int32_t precision, int32_t net, const float* weights, const EjRollout* b,
                                    void* workspace, uint32_t shuffle_ctr, int32_t minibatch,
                                    const double* moments, float* grad, double* stats_out, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = check_common(p, pp, T, hidden, &lay, &kp);
    if (st != EJ_OK) return st;
    if (precision != EJ_FP32 && precision != EJ_BF16) return fail(EJ_ERR_ARG, "unknown precision %d", precision);
    if (net != EJ_NET_POP && net != EJ_NET_GOV) return fail(EJ_ERR_ARG, "unknown network %d", net);
    if (!b || !workspace || !weights || !grad || !moments) return fail(EJ_ERR_ARG, "NULL argument");
    if ((st = check_rollout(b, net, false, true)) != EJ_OK) return st;
    if ((st = check_grad_shape(kp, hidden, precision, net)) != EJ_OK) return st;
    if ((uintptr_t)workspace % 256 || (uintptr_t)weights % 16) return fail(EJ_ERR_ARG, "misaligned buffer");
    if (minibatch < 0 || minibatch >= pp->minibatches) return fail(EJ_ERR_ARG, "minibatch out of range");
    const Ws W = ws_layout(kp, pp, T, hidden);
    char* ws = (char*)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    double* stats = (double*)(ws + W.stats[net]);
    st = minibatch_grad(kp, pp, T, hidden, precision, net, weights, b, ws, W, shuffle_ctr, minibatch, grad, stats, s,
                        moments);
    if (st != EJ_OK) return st;
    if (stats_out) {
        if (cudaMemcpyAsync(stats_out, stats, sizeof(double) * ST_COUNT_, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(EJ_ERR_CUDA, "stats copy failed");
    }
    return EJ_OK;
}

ej_status adam_step(uint64_t n, float* params, const float* grad, float* m, float* v, int32_t step,
                    float lr, float beta1, float beta2, float eps, void* stream) {
    if (!params || !grad || !m || !v) return fail(EJ_ERR_ARG, "NULL argument");
    if (step < 1) return fail(EJ_ERR_ARG, "step counts from 1");
    return launch_adam(params, grad, m, v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream);
}

ej_status ppo_update(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                     int32_t precision, float* pop_w, float* gov_w, float* pop_m, float* pop_v,
                     float* gov_m, float* gov_v, int32_t adam_steps_done, uint32_t update_index,
                     const EjRollout* b, void* workspace, float* stats_out, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = check_common(p, pp, T, hidden, &lay, &kp);
    if (st != EJ_OK) return st;
    if (precision != EJ_FP32 && precision != EJ_BF16) return fail(EJ_ERR_ARG, "unknown precision %d", precision);
    if (!pop_w || !gov_w || !pop_m || !pop_v || !gov_m || !gov_v || !b || !workspace)
        return fail(EJ_ERR_ARG, "NULL argument");
    if ((st = check_rollout(b, -1, true, true)) != EJ_OK) return st;
    if ((st = check_grad_shape(kp, hidden, precision, -1)) != EJ_OK) return st;
    if ((uintptr_t)workspace % 256 || (uintptr_t)pop_w % 16 || (uintptr_t)gov_w % 16)
        return fail(EJ_ERR_ARG, "misaligned buffer");
    const Ws W = ws_layout(kp, pp, T, hidden);
    char* ws = (char*)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ppo_advantages(p, pp, T, b, workspace, stream)) != EJ_OK) return st;
    double* totals = (double*)(ws + W.totals);
    if (cudaMemsetAsync(totals, 0, sizeof(double) * 2 * ST_COUNT_, s) != cudaSuccess)
        return fail(EJ_ERR_CUDA, "memset failed");
    float* w[2] = {pop_w, gov_w};
    float* mm[2] = {pop_m, gov_m};
    float* vv[2] = {pop_v, gov_v};
    int step = adam_steps_done;
    for (int ep = 0; ep < pp->epochs; ++ep) {
        const uint32_t ctr = update_index * (uint32_t)pp->epochs + (uint32_t)ep;
        for (int mb = 0; mb < pp->minibatches; ++mb) {
            ++step;
            for (int net = 0; net < 2; ++net) {
                const NetDims d = dims(kp, net);
                const size_t n = net_offsets(d.in, hidden, d.O).total;
                float* grad = (float*)(ws + W.grad[net]);
                double* stats = (double*)(ws + W.stats[net]);
                st = minibatch_grad(kp, pp, T, hidden, precision, net, w[net], b, ws, W, ctr ^ (net ? 0x80000000u : 0u),
                                    mb, grad, stats, s);
                if (st != EJ_OK) return st;
                accumulate_stats_kernel<<<1, 32, 0, s>>>(stats, totals + net * ST_COUNT_);
                if ((st = launch_adam(w[net], grad, mm[net], vv[net], n, pp->lr, pp->beta1, pp->beta2, pp->eps,
                                      step, s)) != EJ_OK)
                    return st;
            }
        }
    }
    if (stats_out) {
        const double rp = (double)T * kp.E * kp.A * pp->epochs, rg = (double)T * kp.E * pp->epochs;
        finalize_stats_kernel<<<1, 32, 0, s>>>(totals, rp, rg, stats_out);
    }
    return cudaGetLastError() == cudaSuccess ? EJ_OK : fail(EJ_ERR_CUDA, "ppo_update launch failed");
}

ej_status ej_ppo_workspace_bytes_agents(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                                        int32_t layout, uint64_t* bytes) {
    if (layout == EJ_NETS_SHARED) return ej_ppo_workspace_bytes(p, pp, T, hidden, bytes);
    Layout lay;
    KParams kp;
    ej_status st = check_common(p, pp, T, hidden, &lay, &kp);
    if (st != EJ_OK) return st;
    if ((st = check_agents(layout, EJ_FP32)) != EJ_OK) return st;
    if (bytes) *bytes = ws_layout(kp, pp, T, hidden, kp.A).total;
    return EJ_OK;
}

ej_status ppo_minibatch_grad_agents(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                                    int32_t precision, int32_t layout, const float* weights, const EjRollout* b,
                                    void* workspace, uint32_t shuffle_ctr, int32_t minibatch, float* grad,
                                    double* stats_out, void* stream) {
    if (layout == EJ_NETS_SHARED)
        return ppo_minibatch_grad(p, pp, T, hidden, precision, EJ_NET_POP, weights, b, workspace, shuffle_ctr,
                                  minibatch, grad, stats_out, stream);
    Layout lay;
    KParams kp;
    ej_status st = check_common(p, pp, T, hidden, &lay, &kp);
    if (st != EJ_OK) return st;
    if ((st = check_agents(layout, precision)) != EJ_OK) return st;
    if (!b || !workspace || !weights || !grad) return fail(EJ_ERR_ARG, "NULL argument");
    if ((st = check_rollout(b, EJ_NET_POP, false, true)) != EJ_OK) return st;
    if ((st = check_grad_shape(kp, hidden, precision, EJ_NET_POP)) != EJ_OK) return st;
    if ((uintptr_t)workspace % 256 || (uintptr_t)weights % 16) return fail(EJ_ERR_ARG, "misaligned buffer");
    if (minibatch < 0 || minibatch >= pp->minibatches) return fail(EJ_ERR_ARG, "minibatch out of range");
    const Ws W = ws_layout(kp, pp, T, hidden, kp.A);
    char* ws = (char*)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    double* stats = (double*)(ws + W.stats[EJ_NET_POP]);
    st = minibatch_grad_agents(kp, pp, T, hidden, layout, weights, b, ws, W, shuffle_ctr, minibatch, grad, stats, s);
    if (st != EJ_OK) return st;
    if (stats_out &&
        cudaMemcpyAsync(stats_out, stats, sizeof(double) * ST_COUNT_, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(EJ_ERR_CUDA, "stats copy failed");
    return EJ_OK;
}

ej_status ppo_update_agents(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden, int32_t precision,
                            int32_t layout, float* pop_w, float* gov_w, float* pop_m, float* pop_v, float* gov_m,
                            float* gov_v, int32_t adam_steps_done, uint32_t update_index, const EjRollout* b,
                            void* workspace, float* stats_out, void* stream) {
    if (layout == EJ_NETS_SHARED)
        return ppo_update(p, pp, T, hidden, precision, pop_w, gov_w, pop_m, pop_v, gov_m, gov_v, adam_steps_done,
                          update_index, b, workspace, stats_out, stream);
    Layout lay;
    KParams kp;
    ej_status st = check_common(p, pp, T, hidden, &lay, &kp);
    if (st != EJ_OK) return st;
    if ((st = check_agents(layout, precision)) != EJ_OK) return st;
    if (!pop_w || !gov_w || !pop_m || !pop_v || !gov_m || !gov_v || !b || !workspace)
        return fail(EJ_ERR_ARG, "NULL argument");
    if ((st = check_rollout(b, -1, true, true)) != EJ_OK) return st;
    if ((st = check_grad_shape(kp, hidden, precision, -1)) != EJ_OK) return st;
    if ((uintptr_t)workspace % 256 || (uintptr_t)pop_w % 16 || (uintptr_t)gov_w % 16)
        return fail(EJ_ERR_ARG, "misaligned buffer");
    const Ws W = ws_layout(kp, pp, T, hidden, kp.A);
    char* ws = (char*)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ppo_advantages(p, pp, T, b, workspace, stream)) != EJ_OK) return st;
    double* totals = (double*)(ws + W.totals);
    if (cudaMemsetAsync(totals, 0, sizeof(double) * 2 * ST_COUNT_, s) != cudaSuccess)
        return fail(EJ_ERR_CUDA, "memset failed");
    const NetDims dp = dims(kp, EJ_NET_POP), dg = dims(kp, EJ_NET_GOV);
    const size_t n_pop = net_offsets(dp.in, hidden, dp.O).total * kp.A, n_gov = net_offsets(dg.in, hidden, dg.O).total;
    int step = adam_steps_done;
    for (int ep = 0; ep < pp->epochs; ++ep) {
        const uint32_t ctr = update_index * (uint32_t)pp->epochs + (uint32_t)ep;
        for (int mb = 0; mb < pp->minibatches; ++mb) {
            ++step;
            // the population's per-agent networks
            float* gp = (float*)(ws + W.grad[EJ_NET_POP]);
            double* sp = (double*)(ws + W.stats[EJ_NET_POP]);
            if ((st = minibatch_grad_agents(kp, pp, T, hidden, layout, pop_w, b, ws, W, ctr, mb, gp, sp, s)) != EJ_OK)
                return st;
            accumulate_stats_kernel<<<1, 32, 0, s>>>(sp, totals);
            if ((st = launch_adam(pop_w, gp, pop_m, pop_v, n_pop, pp->lr, pp->beta1, pp->beta2, pp->eps, step, s)) != EJ_OK)
                return st;
            // the government's shared network, as in ppo_update
            float* gg = (float*)(ws + W.grad[EJ_NET_GOV]);
            double* sg = (double*)(ws + W.stats[EJ_NET_GOV]);
            if ((st = minibatch_grad(kp, pp, T, hidden, precision, EJ_NET_GOV, gov_w, b, ws, W, ctr ^ 0x80000000u,
                                     mb, gg, sg, s)) != EJ_OK)
                return st;
            accumulate_stats_kernel<<<1, 32, 0, s>>>(sg, totals + ST_COUNT_);
            if ((st = launch_adam(gov_w, gg, gov_m, gov_v, n_gov, pp->lr, pp->beta1, pp->beta2, pp->eps, step, s)) != EJ_OK)
                return st;
        }
    }
    if (stats_out) {
        const double rp = (double)T * kp.E * kp.A * pp->epochs, rg = (double)T * kp.E * pp->epochs;
        finalize_stats_kernel<<<1, 32, 0, s>>>(totals, rp, rg, stats_out);
    }
    return cudaGetLastError() == cudaSuccess ? EJ_OK : fail(EJ_ERR_CUDA, "ppo_update_agents launch failed");
}

}  // extern "C"
