// env_step_host: env_step with inputs and outputs in host memory.
//
// The steps run in chunks through two sets of device staging buffers in a
// caller-owned workspace.  Three library-owned streams per device form a
// pipeline: chunk k+1's inputs copy in (host to device) while chunk k runs
// and chunk k-1's outputs copy out (device to host), so the host link and
// the environment kernel overlap.  The streams fork from the caller's stream
// and join back into it, so the whole call is ordered on that stream.
#include <cstring>
#include <mutex>

#include "ej_internal.cuh"

namespace ej {

namespace {

enum { IN_ACT, IN_GU, IN_TB, IN_GOV, OUT_REW, OUT_GREW, OUT_DONE, OUT_OBS, OUT_GOBS, OUT_MASK, N_ARR };

uint64_t up256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// Bytes per step of each array ([n][E][A], [n][E][nb], ...).
void step_bytes(const KParams& kp, uint64_t* b) {
    const uint64_t EA = (uint64_t)kp.E * kp.A;
    b[IN_ACT] = 4 * EA; b[IN_GU] = 4 * EA; b[IN_TB] = 4 * EA; b[IN_GOV] = 4ull * kp.E * kp.nb;
    b[OUT_REW] = 4 * EA; b[OUT_GREW] = 4ull * kp.E; b[OUT_DONE] = (uint64_t)kp.E;
    b[OUT_OBS] = 4 * EA * kp.D; b[OUT_GOBS] = 4ull * kp.E * kp.G; b[OUT_MASK] = 4 * EA * kp.W;
}

// Offsets of buffer set `set` (0, 1) in the workspace; returns the total.
uint64_t ws_offsets(const KParams& kp, int chunk, uint64_t off[2][N_ARR]) {
    uint64_t b[N_ARR];
    step_bytes(kp, b);
    uint64_t o = 0;
    for (int set = 0; set < 2; ++set)
        for (int k = 0; k < N_ARR; ++k) {
            off[set][k] = o;
            o = up256(o + b[k] * (uint64_t)chunk);
        }
    return o;
}

struct HostIoRes {
    bool ready = false;
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    cudaEvent_t fork = nullptr, ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {}, join[3] = {};
    std::mutex call;          // one call at a time per device enqueues on these streams
};

ej_status host_io_resources(HostIoRes** out) {
    static HostIoRes res[kMaxDevices];
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(EJ_ERR_CUDA, "env_step_host: no device");
    std::lock_guard<std::mutex> lock(mu);
    HostIoRes& r = res[dev];
    if (!r.ready) {
        cudaStream_t* ss[3] = {&r.s_in, &r.s_comp, &r.s_out};
        for (cudaStream_t* s : ss)
            if (cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) != cudaSuccess)
                return fail(EJ_ERR_CUDA, "env_step_host: stream creation failed");
        cudaEvent_t* evs[] = {&r.fork, &r.ev_in[0], &r.ev_in[1], &r.ev_comp[0], &r.ev_comp[1],
                              &r.ev_out[0], &r.ev_out[1], &r.join[0], &r.join[1], &r.join[2]};
        for (cudaEvent_t* e : evs)
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess)
                return fail(EJ_ERR_CUDA, "env_step_host: event creation failed");
        r.ready = true;
    }
    *out = &r;
    return EJ_OK;
}

#define EJ_TRY(call, what)                                                                 \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return fail(EJ_ERR_CUDA, "env_step_host: %s: %s", what,   \
                                           cudaGetErrorString(e_));                        \
    } while (0)

}  // namespace

}  // namespace ej

using namespace ej;

extern "C" {

ej_status ej_step_host_workspace_bytes(const EjParams* p, int32_t chunk, uint64_t* bytes) {
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    if (chunk < 1) return fail(EJ_ERR_ARG, "chunk must be >= 1");
    if (!bytes) return fail(EJ_ERR_ARG, "bytes is NULL");
    uint64_t off[2][N_ARR];
    *bytes = ws_offsets(kp, chunk, off);
    return EJ_OK;
}

ej_status env_step_host(const EjParams* p, void* state, int32_t n_steps, int32_t chunk,
                        const int32_t* act, const int32_t* gov_act, const float* gather_u, const uint32_t* tb,
                        float* rew, float* grew, uint8_t* done, float* obs, float* gobs, uint32_t* mask,
                        void* workspace, uint64_t workspace_bytes, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    if (!state || !workspace) return fail(EJ_ERR_ARG, "env_step_host: NULL state or workspace");
    if ((uintptr_t)state % 256 || (uintptr_t)workspace % 256)
        return fail(EJ_ERR_ARG, "env_step_host: state and workspace must be 256-byte aligned");
    if (n_steps < 0) return fail(EJ_ERR_ARG, "n_steps must be >= 0");
    if (chunk < 1) return fail(EJ_ERR_ARG, "chunk must be >= 1");
    if ((gather_u == nullptr) != (tb == nullptr))
        return fail(EJ_ERR_ARG, "gather_u and tb must be both given or both NULL");
    if (!act && gather_u) return fail(EJ_ERR_ARG, "gather_u and tb need act");
    if (chunk > n_steps && n_steps > 0) chunk = n_steps;
    uint64_t off[2][N_ARR];
    const uint64_t need = ws_offsets(kp, chunk, off);
    if (workspace_bytes < need)
        return fail(EJ_ERR_ARG, "env_step_host: workspace of %llu bytes, %llu needed for chunks of %d steps",
                    (unsigned long long)workspace_bytes, (unsigned long long)need, chunk);
    if (n_steps == 0) return EJ_OK;
    HostIoRes* r = nullptr;
    if ((st = host_io_resources(&r)) != EJ_OK) return st;
    std::lock_guard<std::mutex> lock(r->call);
    uint64_t sb[N_ARR];
    step_bytes(kp, sb);
    const void* host_in[4] = {act, gather_u, tb, gov_act};
    void* host_out[6] = {rew, grew, done, obs, gobs, mask};
    char* ws = (char*)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    EJ_TRY(cudaEventRecord(r->fork, s), "fork");
    EJ_TRY(cudaStreamWaitEvent(r->s_in, r->fork, 0), "fork");
    EJ_TRY(cudaStreamWaitEvent(r->s_comp, r->fork, 0), "fork");
    EJ_TRY(cudaStreamWaitEvent(r->s_out, r->fork, 0), "fork");
    const int n_chunks = (n_steps + chunk - 1) / chunk;
    for (int c = 0; c < n_chunks; ++c) {
        const int b = c & 1;
        const int64_t lo = (int64_t)c * chunk;
        const int n = (int)((n_steps - lo) < chunk ? (n_steps - lo) : chunk);
        // inputs of chunk c into set b, once chunk c-2's kernel no longer reads them
        if (c >= 2) EJ_TRY(cudaStreamWaitEvent(r->s_in, r->ev_comp[b], 0), "wait");
        for (int k = 0; k < 4; ++k)
            if (host_in[k])
                EJ_TRY(cudaMemcpyAsync(ws + off[b][k], (const char*)host_in[k] + (uint64_t)lo * sb[k],
                                       (uint64_t)n * sb[k], cudaMemcpyHostToDevice, r->s_in), "input copy");
        EJ_TRY(cudaEventRecord(r->ev_in[b], r->s_in), "record");
        // the steps, once the inputs have landed and chunk c-2's outputs have left set b
        EJ_TRY(cudaStreamWaitEvent(r->s_comp, r->ev_in[b], 0), "wait");
        if (c >= 2) EJ_TRY(cudaStreamWaitEvent(r->s_comp, r->ev_out[b], 0), "wait");
        auto dev = [&](int k, const void* h) -> void* { return h ? (void*)(ws + off[b][k]) : nullptr; };
        st = env_step(p, state, n, (const int32_t*)dev(IN_ACT, act), (const int32_t*)dev(IN_GOV, gov_act),
                      (const float*)dev(IN_GU, gather_u), (const uint32_t*)dev(IN_TB, tb),
                      (float*)dev(OUT_REW, rew), (float*)dev(OUT_GREW, grew), (uint8_t*)dev(OUT_DONE, done),
                      (float*)dev(OUT_OBS, obs), (float*)dev(OUT_GOBS, gobs), (uint32_t*)dev(OUT_MASK, mask),
                      r->s_comp);
        if (st != EJ_OK) return st;
        EJ_TRY(cudaEventRecord(r->ev_comp[b], r->s_comp), "record");
        // outputs of chunk c back to the host
        EJ_TRY(cudaStreamWaitEvent(r->s_out, r->ev_comp[b], 0), "wait");
        for (int k = 0; k < 6; ++k)
            if (host_out[k])
                EJ_TRY(cudaMemcpyAsync((char*)host_out[k] + (uint64_t)lo * sb[OUT_REW + k], ws + off[b][OUT_REW + k],
                                       (uint64_t)n * sb[OUT_REW + k], cudaMemcpyDeviceToHost, r->s_out),
                       "output copy");
        EJ_TRY(cudaEventRecord(r->ev_out[b], r->s_out), "record");
    }
    cudaStream_t own[3] = {r->s_in, r->s_comp, r->s_out};
    for (int k = 0; k < 3; ++k) {
        EJ_TRY(cudaEventRecord(r->join[k], own[k]), "join");
        EJ_TRY(cudaStreamWaitEvent(s, r->join[k], 0), "join");
    }
    return EJ_OK;
}

}  // extern "C"
