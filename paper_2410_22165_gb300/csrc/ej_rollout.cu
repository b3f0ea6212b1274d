// C ABI of the policy side: network sizes, policy_forward (single and
// segmented launches), rollout and split rollouts.
#include <cstring>
#include <mutex>

#include "ej_internal.cuh"
#include "ej_policy.cuh"

namespace ej {

static ej_status net_shape(const EjParams* p, const KParams& kp, int net, int hidden, int* in,
                           int* O, int* heads, int* head) {
    if (hidden < 32 || hidden > 256 || hidden % 32) return fail(EJ_ERR_UNSUPPORTED, "hidden must be a multiple of 32 in [32, 256]");
    if (net == EJ_NET_POP) { *in = kp.D; *heads = 1; *head = kp.nA; }
    else if (net == EJ_NET_GOV) { *in = kp.G; *heads = kp.nb; *head = p->tax_levels; }
    else return fail(EJ_ERR_ARG, "unknown network %d", net);
    *O = *heads * *head;
    return EJ_OK;
}

static ej_status make_args(const EjParams* p, const KParams& kp, const Layout& lay, const void* state,
                           int net, int hidden, const float* weights, const float* obs,
                           const uint32_t* mask, const float* u, int32_t* act, float* logp,
                           float* value, float* entropy, float* logits, PolicyArgs* a) {
    int in, O, heads, head;
    ej_status st = net_shape(p, kp, net, hidden, &in, &O, &heads, &head);
    if (st != EJ_OK) return st;
    if (!state || !weights || !obs || !value) return fail(EJ_ERR_ARG, "state, weights, obs and value are required");
    if (act && !logp) return fail(EJ_ERR_ARG, "sampling needs logp");
    if ((uintptr_t)weights % 16) return fail(EJ_ERR_ARG, "weights must be 16-byte aligned");
    memset(a, 0, sizeof *a);
    a->rows = net == EJ_NET_POP ? kp.E * kp.A : kp.E;
    a->per_env = net == EJ_NET_POP ? kp.A : 1;
    a->in_dim = in;
    a->in_pad = (in + 3) & ~3;
    a->H = hidden;
    a->O = O;
    a->n_heads = heads;
    a->head = head;
    a->W = (net == EJ_NET_POP && mask) ? kp.W : 0;
    a->stream_id = net == EJ_NET_POP ? 0 : 1;
    a->weights = weights;
    a->x = obs;
    a->mask = a->W ? mask : nullptr;
    a->u = u;
    const DevState s = state_pointers(lay, const_cast<void*>(state));
    a->gstep = s.gstep;
    a->key = s.key;
    a->act = act;
    a->logp = logp;
    a->value = value;
    a->entropy = entropy;
    a->logits = logits;
    return EJ_OK;
}

// Per-agent population networks (Section 5): strides of the actor and the
// critic between the agents' parameter vectors.
static ej_status agent_layout(const EjParams* p, const KParams& kp, int layout, int hidden, int precision,
                              PolicyArgs* a) {
    if (layout == EJ_NETS_SHARED) return EJ_OK;
    if (layout != EJ_NETS_INDEPENDENT && layout != EJ_NETS_CTDE) return fail(EJ_ERR_ARG, "unknown network layout %d", layout);
    if (precision != EJ_FP32 && precision != EJ_BF16) return fail(EJ_ERR_ARG, "unknown precision %d", precision);
    int in, O, heads, head;
    ej_status st = net_shape(p, kp, EJ_NET_POP, hidden, &in, &O, &heads, &head);
    if (st != EJ_OK) return st;
    const size_t n = net_offsets(in, hidden, O).total;
    a->agents = kp.A;
    a->actor_stride = n;
    a->critic_stride = layout == EJ_NETS_INDEPENDENT ? n : 0;
    return EJ_OK;
}

static ej_status launch_policy(const PolicyArgs& a, int precision, cudaStream_t stream) {
    if (precision == EJ_FP32) return launch_policy_fp32(a, stream);
    if (precision == EJ_BF16) return launch_policy_bf16(a, stream);
    return fail(EJ_ERR_UNSUPPORTED, "precision %d is not available", precision);
}

}  // namespace ej

using namespace ej;

extern "C" {

ej_status ej_net_floats(const EjParams* p, int32_t net, int32_t hidden, uint64_t* n_floats) {
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    int in, O, heads, head;
    st = net_shape(p, kp, net, hidden, &in, &O, &heads, &head);
    if (st != EJ_OK) return st;
    if (n_floats) *n_floats = net_offsets(in, hidden, O).total;
    return EJ_OK;
}

ej_status policy_forward(const EjParams* p, const void* state, int32_t net, int32_t hidden,
                         int32_t precision, const float* weights, const float* obs,
                         const uint32_t* mask, const float* u, int32_t* act, float* logp,
                         float* value, float* entropy, float* logits, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    PolicyArgs a;
    st = make_args(p, kp, lay, state, net, hidden, weights, obs, mask, u, act, logp, value, entropy,
                   logits, &a);
    if (st != EJ_OK) return st;
    return launch_policy(a, precision, (cudaStream_t)stream);
}

ej_status policy_forward_agents(const EjParams* p, const void* state, int32_t layout, int32_t hidden,
                                int32_t precision, const float* weights, const float* obs, const uint32_t* mask,
                                const float* u, int32_t* act, float* logp, float* value, float* entropy,
                                float* logits, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    PolicyArgs a;
    st = make_args(p, kp, lay, state, EJ_NET_POP, hidden, weights, obs, mask, u, act, logp, value, entropy,
                   logits, &a);
    if (st != EJ_OK) return st;
    if ((st = agent_layout(p, kp, layout, hidden, precision, &a)) != EJ_OK) return st;
    return launch_policy(a, precision, (cudaStream_t)stream);
}

ej_status policy_segmented(const EjParams* p, int32_t net, int32_t hidden, int32_t precision, int32_t* ok) {
    if (!ok) return fail(EJ_ERR_ARG, "policy_segmented: NULL argument");
    *ok = 0;
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    int in_dim, O, heads, head;
    if ((st = net_shape(p, kp, net, hidden, &in_dim, &O, &heads, &head)) != EJ_OK) return st;
    const int W = net == EJ_NET_POP ? kp.W : 0;
    *ok = precision == EJ_BF16 && hidden == 128 && O <= 96 && in_dim <= 32 && W <= 4 && heads <= EJ_MAX_NB;
    return EJ_OK;
}

ej_status policy_forward_segments(int32_t n_seg, const EjParams* const* params, const void* const* states,
                                  const int32_t* nets, const float* const* weights, int32_t hidden,
                                  int32_t precision, const float* const* obs, const uint32_t* const* mask,
                                  int32_t* const* act, float* const* logp, float* const* value, void* stream) {
    if (n_seg < 1 || !params || !states || !nets || !weights || !obs || !value)
        return fail(EJ_ERR_ARG, "policy_forward_segments: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    PolicyArgs args[EJ_MAX_SEG];
    int n = 0;
    auto flush = [&]() -> ej_status {
        if (n == 0) return EJ_OK;
        bool handled = false;
        if (precision == EJ_BF16) {
            ej_status st = launch_policy_bf16_multi(args, n, s, &handled);
            if (st != EJ_OK) return st;
        }
        for (int q = 0; q < n && !handled; ++q) {
            ej_status st = launch_policy(args[q], precision, s);
            if (st != EJ_OK) return st;
        }
        n = 0;
        return EJ_OK;
    };
    for (int k = 0; k < n_seg; ++k) {
        Layout lay;
        KParams kp;
        ej_status st = derive(params[k], &lay, &kp);
        if (st != EJ_OK) return st;
        if (nets[k] == EJ_NET_GOV && mask && mask[k]) return fail(EJ_ERR_ARG, "policy_forward_segments: the government takes no mask");
        PolicyArgs a;
        st = make_args(params[k], kp, lay, states[k], nets[k], hidden, weights[k], obs[k],
                       mask && nets[k] == EJ_NET_POP ? mask[k] : nullptr, nullptr, act ? act[k] : nullptr,
                       logp ? logp[k] : nullptr, value[k], nullptr, nullptr, &a);
        if (st != EJ_OK) return st;
        // a launch takes at most EJ_MAX_SEG segments of at most EJ_MAX_NET networks
        int nets_in = 0;
        bool known = false;
        for (int q = 0; q < n; ++q) {
            bool first = true;
            for (int r = 0; r < q; ++r)
                if (args[r].weights == args[q].weights && args[r].stream_id == args[q].stream_id) first = false;
            nets_in += first;
            if (args[q].weights == a.weights && args[q].stream_id == a.stream_id) known = true;
        }
        if (n == EJ_MAX_SEG || (!known && nets_in == EJ_MAX_NET))
            if ((st = flush()) != EJ_OK) return st;
        args[n++] = a;
    }
    return flush();
}

}  // extern "C"

namespace {

// T steps of {population policy, government policy, env_step} for the
// environments [e0, e0 + ne) into the rollout buffer's rows of those
// environments, then their bootstrap values, on one stream.
ej_status rollout_range(const EjParams* p, const KParams& kp, const Layout& lay, void* state, int T, int hidden,
                        int precision, const float* pop_weights, const float* gov_weights, const EjRollout* b,
                        int e0, int ne, cudaStream_t s, int layout = EJ_NETS_SHARED) {
    const size_t EA = (size_t)kp.E * kp.A, A = kp.A;
    const DevState ds = state_pointers(lay, state);
    KParams kr = kp;
    kr.e0 = e0;
    kr.ne = ne;
    ej_status st;
    for (int t = 0; t <= T; ++t) {
        const bool last = t == T;
        PolicyArgs pa, ga;
        const size_t r0 = (size_t)e0 * A;          // first population row of the range
        st = make_args(p, kp, lay, state, EJ_NET_POP, hidden, pop_weights, b->obs + (t * EA + r0) * kp.D,
                       b->mask + (t * EA + r0) * kp.W, nullptr, last ? nullptr : b->act + t * EA + r0,
                       last ? nullptr : b->logp + t * EA + r0, b->value + t * EA + r0, nullptr, nullptr, &pa);
        if (st != EJ_OK) return st;
        if ((st = agent_layout(p, kp, layout, hidden, precision, &pa)) != EJ_OK) return st;
        pa.rows = ne * kp.A;
        pa.env0 = e0;
        const size_t g0 = (size_t)t * kp.E + e0;    // first government row of the range
        st = make_args(p, kp, lay, state, EJ_NET_GOV, hidden, gov_weights, b->gobs + g0 * kp.G, nullptr, nullptr,
                       last ? nullptr : b->gact + g0 * kp.nb, last ? nullptr : b->glogp + g0, b->gvalue + g0,
                       nullptr, nullptr, &ga);
        if (st != EJ_OK) return st;
        ga.rows = ne;
        ga.env0 = e0;
        // BF16: population and government networks in one launch where the kernel takes both
        // (shared networks only)
        bool handled = false;
        if (precision == EJ_BF16 && pa.agents == 0) {
            const PolicyArgs both[2] = {pa, ga};
            if ((st = launch_policy_bf16_multi(both, 2, s, &handled)) != EJ_OK) return st;
        }
        if (!handled) {
            if ((st = launch_policy(pa, precision, s)) != EJ_OK) return st;
            if ((st = launch_policy(ga, precision, s)) != EJ_OK) return st;
        }
        if (last) break;
        DevIO io;
        memset(&io, 0, sizeof io);
        io.act = b->act + t * EA;
        io.gov_act = b->gact + (size_t)t * kp.E * kp.nb;
        io.rew = b->rew + t * EA;
        io.grew = b->grew + (size_t)t * kp.E;
        io.done = b->done + (size_t)t * kp.E;
        io.obs = b->obs + (t + 1) * EA * kp.D;
        io.gobs = b->gobs + (size_t)(t + 1) * kp.E * kp.G;
        io.mask = b->mask + (t + 1) * EA * kp.W;
        if ((st = launch_env(kr, lay, ds, io, 1, MODE_AUX_DRAW, 0, s)) != EJ_OK) return st;
    }
    return EJ_OK;
}

// Streams and events for the chains of a split rollout (per device, created
// once; the chains fork from and join back to the caller's stream).
constexpr int EJ_MAX_CHAINS = 4;
struct ChainRes {
    cudaStream_t s[EJ_MAX_CHAINS] = {};
    cudaEvent_t ev[EJ_MAX_CHAINS] = {};
    bool ready = false;
};

ej_status chain_resources(ChainRes** out) {
    static ChainRes res[16];
    static std::mutex mu;                      // first calls from several host threads
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return fail(EJ_ERR_CUDA, "rollout: no device");
    std::lock_guard<std::mutex> lock(mu);
    ChainRes& r = res[dev];
    if (!r.ready) {
        for (int c = 0; c < EJ_MAX_CHAINS; ++c) {
            if (c > 0 && cudaStreamCreateWithFlags(&r.s[c], cudaStreamNonBlocking) != cudaSuccess)
                return fail(EJ_ERR_CUDA, "rollout: stream creation failed");
            if (cudaEventCreateWithFlags(&r.ev[c], cudaEventDisableTiming) != cudaSuccess)
                return fail(EJ_ERR_CUDA, "rollout: event creation failed");
        }
        r.ready = true;
    }
    *out = &r;
    return EJ_OK;
}

}  // namespace

extern "C" {

ej_status rollout_split(const EjParams* p, void* state, int32_t T, int32_t hidden, int32_t precision,
                        const float* pop_weights, const float* gov_weights, const EjRollout* b, int32_t n_chains,
                        void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    if (!b || !state || !pop_weights || !gov_weights) return fail(EJ_ERR_ARG, "rollout: NULL argument");
    if (T < 1) return fail(EJ_ERR_ARG, "rollout: T must be >= 1");
    if (!b->obs || !b->gobs || !b->mask || !b->act || !b->gact || !b->logp || !b->glogp ||
        !b->value || !b->gvalue || !b->rew || !b->grew || !b->done)
        return fail(EJ_ERR_ARG, "rollout: every buffer is required");
    if ((uintptr_t)state % 256) return fail(EJ_ERR_ARG, "state must be 256-byte aligned");
    if (n_chains < 1 || n_chains > EJ_MAX_CHAINS) return fail(EJ_ERR_ARG, "rollout: 1 to %d chains", EJ_MAX_CHAINS);
    if (n_chains > kp.E) n_chains = kp.E;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_chains == 1) return rollout_range(p, kp, lay, state, T, hidden, precision, pop_weights, gov_weights, b, 0,
                                            kp.E, s);
    ChainRes* r = nullptr;
    if ((st = chain_resources(&r)) != EJ_OK) return st;
    if (cudaEventRecord(r->ev[0], s) != cudaSuccess) return fail(EJ_ERR_CUDA, "rollout: event record failed");
    for (int c = 1; c < n_chains; ++c)
        if (cudaStreamWaitEvent(r->s[c], r->ev[0], 0) != cudaSuccess) return fail(EJ_ERR_CUDA, "rollout: fork failed");
    for (int c = 0; c < n_chains; ++c) {
        const int e0 = (int)((int64_t)kp.E * c / n_chains), e1 = (int)((int64_t)kp.E * (c + 1) / n_chains);
        st = rollout_range(p, kp, lay, state, T, hidden, precision, pop_weights, gov_weights, b, e0, e1 - e0,
                           c == 0 ? s : r->s[c]);
        if (st != EJ_OK) return st;
    }
    for (int c = 1; c < n_chains; ++c) {
        if (cudaEventRecord(r->ev[c], r->s[c]) != cudaSuccess || cudaStreamWaitEvent(s, r->ev[c], 0) != cudaSuccess)
            return fail(EJ_ERR_CUDA, "rollout: join failed");
    }
    return EJ_OK;
}

ej_status rollout_agents(const EjParams* p, void* state, int32_t T, int32_t hidden, int32_t precision,
                         int32_t layout, const float* pop_weights, const float* gov_weights, const EjRollout* b,
                         void* stream) {
    if (layout == EJ_NETS_SHARED) return rollout(p, state, T, hidden, precision, pop_weights, gov_weights, b, stream);
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    if (!b || !state || !pop_weights || !gov_weights) return fail(EJ_ERR_ARG, "rollout: NULL argument");
    if (T < 1) return fail(EJ_ERR_ARG, "rollout: T must be >= 1");
    if (!b->obs || !b->gobs || !b->mask || !b->act || !b->gact || !b->logp || !b->glogp ||
        !b->value || !b->gvalue || !b->rew || !b->grew || !b->done)
        return fail(EJ_ERR_ARG, "rollout: every buffer is required");
    if ((uintptr_t)state % 256) return fail(EJ_ERR_ARG, "state must be 256-byte aligned");
    PolicyArgs probe;
    memset(&probe, 0, sizeof probe);
    if ((st = agent_layout(p, kp, layout, hidden, precision, &probe)) != EJ_OK) return st;
    return rollout_range(p, kp, lay, state, T, hidden, precision, pop_weights, gov_weights, b, 0, kp.E,
                         (cudaStream_t)stream, layout);
}

ej_status rollout(const EjParams* p, void* state, int32_t T, int32_t hidden, int32_t precision,
                  const float* pop_weights, const float* gov_weights, const EjRollout* b, void* stream) {
    // two chains from 2048 environments: one chain's env_step fills the SMs that the
    // other's policy launch leaves idle at its start and end (E = 4096 x A = 100, BF16:
    // 211.8 -> 203.4 us per step; three or four chains: 219-221 us)
    const int chains = p && p->E >= 2048 ? 2 : 1;
    return rollout_split(p, state, T, hidden, precision, pop_weights, gov_weights, b, chains, stream);
}

}  // extern "C"
