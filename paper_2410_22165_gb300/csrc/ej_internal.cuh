// Internal declarations of the CUDA library (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/econojax.h"

namespace ej {

// Kernel-side copy of the parameters, with the derived sizes.
struct KParams {
    int E, A, A_s, R, P, nb, L, nA, D, G, W, M, cap;
    int e0, ne;                 // environments [e0, e0 + ne) of a launch (default: all)
    int T_ep, T_tax, expire, max_orders, Rk, Rd, allow_noop, gov_enabled, tax_levels;
    float start_coin, ome, omega, lg, lc, lt, craft_coin, gather_rho, tick;
    float skill_gain, skill_max;   // skill improvement (0: off)
    int skill_init;                // 0 U[0,1); 1 Irwin-Hall around 1
    float price[EJ_MAX_P];      // tick * ticks[p], rounded once to float
    int ticks[EJ_MAX_P];
    float th[EJ_MAX_NB];        // bracket edges (nb - 1 used)
};

// Device pointers of every state field.
struct DevState {
    float* coin; int* esc; float* income; float* uprev; int* nord; int* counts; float* sc;
    int* inv; int* inve; float* sg;
    int* t; uint32_t* gstep; uint32_t* episode; int* pop; float* rates; float* ugprev;
    int* lvl; uint32_t* book; uint32_t* key;
};

struct DevIO {
    const int32_t* act; const int32_t* gov_act; const float* gather_u; const uint32_t* tb;
    float* rew; float* grew; uint8_t* done; float* obs; float* gobs; uint32_t* mask;
    const int32_t* pop_sizes;   // env_reset only
};

struct Layout {
    EjSizes sizes;
    uint64_t off[EJ_F_COUNT_];
    uint64_t count[EJ_F_COUNT_];
    int32_t esz[EJ_F_COUNT_];
};

// Validates the parameters and computes sizes, layout and kernel parameters.
ej_status derive(const EjParams* p, Layout* lay, KParams* kp);
DevState state_pointers(const Layout& lay, void* base);

// Records the error message of the calling thread and returns s.
ej_status fail(ej_status s, const char* fmt, ...);

// Per-device launch configuration.  cudaFuncSetAttribute acts on the device
// that is current when it is called, so the dynamic shared-memory size a
// kernel has been opened up to is remembered per device (under a lock: host
// threads may launch concurrently).
constexpr int kMaxDevices = 64;

class SmemOptIn {
 public:
    // Raises `kernel`'s dynamic shared-memory limit on the current device to
    // at least `bytes` (once per device and size).
    ej_status ensure(const void* kernel, size_t bytes) {
        int dev = 0;
        cudaError_t err = cudaGetDevice(&dev);
        if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(err));
        if (dev < 0 || dev >= kMaxDevices) return fail(EJ_ERR_UNSUPPORTED, "device %d: at most %d devices", dev, kMaxDevices);
        std::lock_guard<std::mutex> lock(mu_);
        if (bytes_[dev] >= bytes) return EJ_OK;
        err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (err != cudaSuccess) return fail(EJ_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(err));
        bytes_[dev] = bytes;
        return EJ_OK;
    }

 private:
    std::mutex mu_;
    size_t bytes_[kMaxDevices] = {};
};

// Streaming multiprocessors of the current device (queried once per device;
// at least 1).  Grids are sized in multiples of it.
int device_sms();

// Launchers (ej_env.cu; the 2-resource instantiations with 5, 10 and 20 price levels in
// ej_env_r2p5.cu, ej_env_r2p10.cu, ej_env_r2p20.cu).
enum : int { MODE_RESET = 1, MODE_POP_DRAW = 2, MODE_GOV_DRAW = 4, MODE_AUX_DRAW = 8 };
ej_status launch_env(const KParams& kp, const Layout& lay, const DevState& st, const DevIO& io,
                     int n_steps, int mode, uint64_t seed, cudaStream_t stream);
ej_status launch_env_r2p5(const KParams& kp, const Layout& lay, const DevState& st, const DevIO& io,
                          int n_steps, int mode, uint64_t seed, cudaStream_t stream);
ej_status launch_env_r2p10(const KParams& kp, const Layout& lay, const DevState& st, const DevIO& io,
                           int n_steps, int mode, uint64_t seed, cudaStream_t stream);
ej_status launch_env_r2p20(const KParams& kp, const Layout& lay, const DevState& st, const DevIO& io,
                           int n_steps, int mode, uint64_t seed, cudaStream_t stream);
ej_status launch_fill_draws(const KParams& kp, uint64_t seed, uint32_t g0, int n_steps,
                            int32_t* act, float* gather_u, uint32_t* tb, float* policy_u,
                            int32_t* gov_act, cudaStream_t stream);

// Threads of the CTA that runs one environment of A agents.
inline int env_threads(int A) {
    int nt = 32;
    while (nt < A) nt <<= 1;
    return nt;
}

// Shared-memory carve-up of one environment CTA (host and device agree).
struct SmemLayout {
    uint32_t inv, inve, sg, book, lvl, kb, fl, stat, alias, total;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline SmemLayout smem_layout(int NT, int R, int P, int L, int cap, int M, int D) {
    SmemLayout s;
    uint32_t b = 0;
    s.inv = b;   b = align16(b + 4u * R * NT);
    s.inve = b;  b = align16(b + 4u * R * NT);
    s.sg = b;    b = align16(b + 4u * R * NT);
    s.book = b;  b = align16(b + 8u * cap);   // two buffers
    s.lvl = b;   b = align16(b + 4u * (9u * L + 9u));
    s.kb = b;    b = align16(b + 4u * (R + 2u * R * P));
    const uint32_t nw = NT / 32;
    s.fl = b;    b = align16(b + 4u * (EJ_MAX_NB + 4u * R + nw * (M + 1u) + (M + 1u) + 3u * M + 16u + EJ_MAX_ORDERS + 1u));
    s.stat = b;  b = align16(b + 4u * M * NT);   // government statistics being sorted (own region: the
                                                 // sorts overlap the next step's first phase)
    s.alias = b;
    // phase A: new-order keys, sorted new orders, per-agent integer deltas, tax
    uint32_t a = align16(8u * NT) + align16(4u * NT) + 4u * align16(4u * NT) +
                 2u * align16(4u * R * NT) + align16(4u * NT);
    const uint32_t stage_nt = NT >= 256 ? NT / 2 : NT;
    uint32_t c = 4u * stage_nt * D;          // phase C: observation staging (half of the warps at a time from 256 threads)
    uint32_t m = a > c ? a : c;
    b = align16(b + m);
    s.total = b;
    return s;
}

// Philox-4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// multiplies with a Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ float u01(uint32_t x) {
    return __uint2float_rn(x >> 8) * 5.9604644775390625e-08f;   // * 2^-24, exact
}

__device__ __forceinline__ int below(uint32_t x, int n) { return (int)__umulhi(x, (uint32_t)n); }

}  // namespace ej
