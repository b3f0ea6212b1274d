// ppo_minibatch_grad_static: the PPO minibatch gradient with its scratch
// memory in a fixed array that the library itself holds, for callers that
// cannot allocate device memory.
//
// Such callers exist: hosts whose device memory is owned by another runtime's
// pool allocator that does not hand out extra buffers, plain C programs
// embedding this library with no device allocator of their own, and service
// loops that must not allocate once running.  They can pass their inputs and
// outputs but not a workspace.
//
// The scratch is one file-scope __device__ array of SCRATCH_BYTES (48 MiB),
// which every GPU that loads the library holds until the process exits.  All
// calls share it and it keeps the previous call's contents; everything that
// must start at zero is cleared by the call itself.  Calls that overlap on the
// GPU (different streams, or different host threads) race on the array:
// serialise them.
#include <cstring>
#include <mutex>

#include "ej_internal.cuh"
#include "ej_ppo.cuh"

namespace ej {

namespace {

constexpr size_t SCRATCH_BYTES = 48ull << 20;
constexpr int STATIC_CHUNKS = 16;       // split-K chunks of the weight gradients
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};

uint64_t up256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// Device address of the scratch array for the current device.  On the first
// call for a device, with that device current, it is looked up with
// cudaGetSymbolAddress; that first call therefore must not happen inside a
// stream capture.  (In host code the array's name is only a host-side
// stand-in and must never be passed to a kernel.)
ej_status scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(err));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(EJ_ERR_UNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        err = cudaGetSymbolAddress(&p, g_scratch);
        if (err != cudaSuccess || !p)
            return fail(EJ_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(err));
        g_scratch_ptr[dev] = p;
    }
    *out = (unsigned char*)g_scratch_ptr[dev];
    return EJ_OK;
}

int domain_bits(uint64_t N) {
    int b = 2;
    while ((1ull << b) < N) ++b;
    return b;
}

}  // namespace

}  // namespace ej

using namespace ej;

extern "C" ej_status ppo_minibatch_grad_static(const EjParams* p, const EjPpoParams* pp, int32_t T,
                                               int32_t hidden, int32_t precision, int32_t net,
                                               const float* weights, const EjRollout* b,
                                               uint32_t shuffle_ctr, int32_t minibatch, float* grad,
                                               double* stats_out, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    if (!pp) return fail(EJ_ERR_ARG, "ppo params is NULL");
    if (T < 1) return fail(EJ_ERR_ARG, "T must be >= 1");
    if (pp->minibatches < 1) return fail(EJ_ERR_ARG, "minibatches must be >= 1");
    if (hidden < 32 || hidden > 128 || hidden % 32) return fail(EJ_ERR_UNSUPPORTED, "hidden in {32, 64, 96, 128}");
    if (precision != EJ_FP32) return fail(EJ_ERR_UNSUPPORTED, "precision %d not available", precision);
    if (net != EJ_NET_POP && net != EJ_NET_GOV) return fail(EJ_ERR_ARG, "unknown network %d", net);
    if (!b || !weights || !grad) return fail(EJ_ERR_ARG, "NULL argument");
    if ((uintptr_t)weights % 16) return fail(EJ_ERR_ARG, "weights must be 16-byte aligned");
    if (minibatch < 0 || minibatch >= pp->minibatches) return fail(EJ_ERR_ARG, "minibatch out of range");
    const int H = hidden;
    const bool pop = net == EJ_NET_POP;
    const int in = pop ? kp.D : kp.G, heads = pop ? 1 : kp.nb, head = pop ? kp.nA : kp.tax_levels;
    const int O = heads * head;
    if (in > 128 || O > 128) return fail(EJ_ERR_UNSUPPORTED, "inputs and logits must be <= 128");
    const int rows_per_step = pop ? kp.E * kp.A : kp.E;
    const uint64_t N = (uint64_t)T * rows_per_step;
    if ((uint64_t)pp->minibatches > N)
        return fail(EJ_ERR_ARG, "%d minibatches exceed the network's %llu rows", pp->minibatches, (unsigned long long)N);
    const uint64_t count_max = (N + pp->minibatches - 1) / pp->minibatches;
    const uint64_t row_floats = in + 8ull * H + O + 1;
    // scratch layout: adv, ret, stats, transposed weights, per-row buffers, partials
    uint64_t o = 0;
    const uint64_t o_adv = o;   o = up256(o + 4 * N);
    const uint64_t o_ret = o;   o = up256(o + 4 * N);
    const uint64_t o_stats = o; o = up256(o + 8 * ST_COUNT_);
    const uint64_t o_wt3 = o;   o = up256(o + 4ull * O * H);
    const uint64_t o_wt2 = o;   o = up256(o + 4ull * H * H);
    const uint64_t o_wv2 = o;   o = up256(o + 4ull * H * H);
    const uint64_t o_rows = o;  o = up256(o + 4ull * row_floats * count_max);
    const size_t stride = wg_stride(in, H, O);
    const uint64_t o_part = o;  o = up256(o + 4ull * 6 * STATIC_CHUNKS * stride);
    if (o > SCRATCH_BYTES)
        return fail(EJ_ERR_UNSUPPORTED,
                    "ppo_minibatch_grad_static: this minibatch needs %llu bytes of scratch but the static "
                    "array holds %llu (rollout of %llu rows, minibatch of %llu rows); use ppo_minibatch_grad "
                    "with a caller-allocated workspace",
                    (unsigned long long)o, (unsigned long long)SCRATCH_BYTES, (unsigned long long)N,
                    (unsigned long long)count_max);
    if ((st = check_rollout(b, net, true, true)) != EJ_OK) return st;
    unsigned char* sc = nullptr;
    if ((st = scratch_for_current_device(&sc)) != EJ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float* adv = (float*)(sc + o_adv);
    float* ret = (float*)(sc + o_ret);
    // advantages of this network only
    st = pop ? launch_gae(b->rew, b->value, b->done, T, kp.E * kp.A, kp.A, pp->gamma, pp->lam, adv, ret, s)
             : launch_gae(b->grew, b->gvalue, b->done, T, kp.E, 1, pp->gamma, pp->lam, adv, ret, s);
    if (st != EJ_OK) return st;
    const NetOffsets off = net_offsets(in, H, O);
    FbArgs fa;
    memset(&fa, 0, sizeof fa);
    fa.mb.lo = (int)((N * minibatch) / pp->minibatches);
    fa.mb.count = (int)((N * (minibatch + 1)) / pp->minibatches) - fa.mb.lo;
    fa.mb.N = (uint32_t)N;
    fa.mb.bits = domain_bits(N);
    fa.mb.k0 = (uint32_t)pp->seed;
    fa.mb.k1 = (uint32_t)(pp->seed >> 32);
    fa.mb.ctr = shuffle_ctr;
    fa.in_dim = in; fa.in_pad = (in + 3) & ~3; fa.H = H; fa.O = O;
    fa.n_heads = heads; fa.head = head; fa.W = pop ? kp.W : 0;
    fa.clip = pp->clip; fa.vf_coef = pp->vf_coef; fa.vclip = pp->vclip; fa.ent_coef = pp->ent_coef;
    fa.weights = weights;
    if (pop) { fa.x = b->obs; fa.mask = b->mask; fa.act = b->act; fa.logp_old = b->logp; fa.v_old = b->value; }
    else { fa.x = b->gobs; fa.mask = nullptr; fa.act = b->gact; fa.logp_old = b->glogp; fa.v_old = b->gvalue; }
    fa.adv = adv;
    fa.ret = ret;
    fa.w3t = (float*)(sc + o_wt3); fa.w2t = (float*)(sc + o_wt2); fa.v2t = (float*)(sc + o_wv2);
    fa.stats = (double*)(sc + o_stats);      // cleared by the gradient launch itself
    const uint64_t R = (uint64_t)fa.mb.count;
    float* rb = (float*)(sc + o_rows);
    // hidden-width arrays first: each starts on a 16-byte boundary (H is a multiple of 32)
    fa.ws_h1 = rb; rb += R * H;
    fa.ws_h2 = rb; rb += R * H;
    fa.ws_g1 = rb; rb += R * H;
    fa.ws_g2 = rb; rb += R * H;
    fa.ws_dz2 = rb; rb += R * H;
    fa.ws_dz1 = rb; rb += R * H;
    fa.ws_dy2 = rb; rb += R * H;
    fa.ws_dy1 = rb; rb += R * H;
    fa.ws_x = rb; rb += R * in;
    fa.ws_dl = rb; rb += R * O;
    fa.ws_dv = rb;
    WgJobs jobs;
    memset(&jobs, 0, sizeof jobs);
    const float* A_[6] = {fa.ws_x, fa.ws_h1, fa.ws_h2, fa.ws_x, fa.ws_g1, fa.ws_g2};
    const float* B_[6] = {fa.ws_dz1, fa.ws_dz2, fa.ws_dl, fa.ws_dy1, fa.ws_dy2, fa.ws_dv};
    const int m_[6] = {in, H, H, in, H, H}, n_[6] = {H, H, O, H, H, 1};
    const size_t wo[6] = {off.W1, off.W2, off.W3, off.V1, off.V2, off.V3};
    const size_t bo[6] = {off.b1, off.b2, off.b3, off.c1, off.c2, off.c3};
    for (int q = 0; q < 6; ++q) {
        jobs.job[q].A = A_[q]; jobs.job[q].B = B_[q]; jobs.job[q].lda = m_[q]; jobs.job[q].ldb = n_[q];
        jobs.job[q].m = m_[q]; jobs.job[q].n = n_[q];
        jobs.job[q].w_off = (long long)wo[q]; jobs.job[q].b_off = (long long)bo[q];
    }
    if (cudaMemsetAsync(grad, 0, sizeof(float) * off.total, s) != cudaSuccess)
        return fail(EJ_ERR_CUDA, "memset of the gradient failed");
    st = launch_minibatch_grad(fa, jobs, 6, (float*)(sc + o_part), stride, STATIC_CHUNKS, weights + off.W2,
                               weights + off.W3, weights + off.V2, grad, s);
    if (st != EJ_OK) return st;
    st = launch_minibatch_loss(fa.stats, fa.mb.count, nullptr, pp->vf_coef, pp->ent_coef, s);
    if (st != EJ_OK) return st;
    if (stats_out &&
        cudaMemcpyAsync(stats_out, fa.stats, sizeof(double) * ST_COUNT_, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(EJ_ERR_CUDA, "stats copy failed");
    return EJ_OK;
}
