// C ABI of the environment: parameter defaults and validation, the state
// layout, and the entry points declared in include/econojax.h.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "ej_internal.cuh"

namespace ej {

static thread_local char g_err[512] = "";

ej_status fail(ej_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

int device_sms() {
    static std::mutex mu;
    static int sms[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
    std::lock_guard<std::mutex> lock(mu);
    if (sms[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        sms[dev] = n;
    }
    return sms[dev];
}

static uint64_t align256(uint64_t x) { return (x + 255u) & ~uint64_t(255u); }

ej_status derive(const EjParams* p, Layout* lay, KParams* kp) {
    if (!p) return fail(EJ_ERR_ARG, "params is NULL");
    if (p->E < 1) return fail(EJ_ERR_ARG, "E must be >= 1 (got %d)", p->E);
    if (p->A < 1 || p->A > EJ_MAX_A) return fail(EJ_ERR_UNSUPPORTED, "A must be in [1, %d] (got %d)", EJ_MAX_A, p->A);
    if (p->R < 1 || p->R > EJ_MAX_R) return fail(EJ_ERR_UNSUPPORTED, "R must be in [1, %d]", EJ_MAX_R);
    if (p->P < 1 || p->P > EJ_MAX_P) return fail(EJ_ERR_UNSUPPORTED, "P must be in [1, %d]", EJ_MAX_P);
    if (p->nb < 1 || p->nb > EJ_MAX_NB) return fail(EJ_ERR_UNSUPPORTED, "nb must be in [1, %d]", EJ_MAX_NB);
    if (p->T_ep < 1 || p->T_ep > 65535) return fail(EJ_ERR_UNSUPPORTED, "T_ep must be in [1, 65535]");
    if (p->T_tax < 1) return fail(EJ_ERR_ARG, "T_tax must be >= 1");
    if (p->expire < 1) return fail(EJ_ERR_ARG, "expire must be >= 1");
    if (p->max_orders < 0 || p->max_orders > EJ_MAX_ORDERS)
        return fail(EJ_ERR_UNSUPPORTED, "max_orders must be in [0, %d]", EJ_MAX_ORDERS);
    if (p->Rk < 0 || p->Rd < 0 || p->Rd > p->R) return fail(EJ_ERR_ARG, "need Rk >= 0 and 0 <= Rd <= R");
    if (p->tax_levels < 2) return fail(EJ_ERR_ARG, "tax_levels must be >= 2");
    const int nA = 2 + p->R + 2 * p->R * p->P;
    const int L = 2 * p->R * p->P;
    if (nA > EJ_MAX_ACTIONS) return fail(EJ_ERR_UNSUPPORTED, "2 + R + 2RP must be <= %d", EJ_MAX_ACTIONS);
    if (L > EJ_MAX_LEVELS) return fail(EJ_ERR_UNSUPPORTED, "2RP must be <= %d", EJ_MAX_LEVELS);
    if (!(p->eta >= 0.0f) || p->eta == 1.0f) return fail(EJ_ERR_ARG, "eta must be >= 0 and != 1");
    if (!(p->price_tick > 0.0f)) return fail(EJ_ERR_ARG, "price_tick must be > 0");
    for (int q = 0; q < p->P; ++q) {
        if (p->price_ticks[q] < 1 || p->price_ticks[q] > 1000000)
            return fail(EJ_ERR_ARG, "price_ticks[%d] out of range", q);
        if (q && p->price_ticks[q] <= p->price_ticks[q - 1])
            return fail(EJ_ERR_ARG, "price_ticks must be strictly ascending");
    }
    for (int b = 1; b + 1 < p->nb; ++b)
        if (!(p->thresholds[b] > p->thresholds[b - 1])) return fail(EJ_ERR_ARG, "thresholds must ascend");
    if (!(p->skill_gain >= 0.0f) || !(p->skill_max > 0.0f)) return fail(EJ_ERR_ARG, "need skill_gain >= 0 and skill_max > 0");
    if (p->skill_init != 0 && p->skill_init != 1) return fail(EJ_ERR_ARG, "skill_init must be 0 or 1");

    const int A_s = (p->A + 3) & ~3;
    const int D = 8 + 7 * p->R + p->nb;
    const int G = 3 * 3 + p->nb + 2;
    const int W = (nA + 31) / 32;
    const int M = 3;          // statistics metrics: total coin, period earnings, labor
    const int cap = p->A * (p->max_orders > 0 ? p->max_orders : 1);
    const int NT = env_threads(p->A);
    const SmemLayout sl = smem_layout(NT, p->R, p->P, L, cap, M, D);
    if (sl.total > 227u * 1024u) return fail(EJ_ERR_UNSUPPORTED, "environment needs %u bytes of shared memory", sl.total);

    Layout L_;
    memset(&L_, 0, sizeof L_);
    const uint64_t E = (uint64_t)p->E;
    struct { int f; uint64_t n; int esz; } fields[] = {
        {EJ_F_COIN, E * A_s, 4}, {EJ_F_ESC, E * A_s, 4}, {EJ_F_INCOME, E * A_s, 4},
        {EJ_F_UPREV, E * A_s, 4}, {EJ_F_NORD, E * A_s, 4}, {EJ_F_COUNTS, E * 3 * A_s, 4},
        {EJ_F_SC, E * A_s, 4}, {EJ_F_INV, E * p->R * A_s, 4}, {EJ_F_INVE, E * p->R * A_s, 4},
        {EJ_F_SG, E * p->R * A_s, 4}, {EJ_F_T, E, 4}, {EJ_F_GSTEP, E, 4}, {EJ_F_EPISODE, E, 4},
        {EJ_F_POP, E, 4}, {EJ_F_RATES, E * EJ_MAX_NB, 4}, {EJ_F_UGPREV, E, 4},
        {EJ_F_LEVEL_COUNT, E * L, 4}, {EJ_F_BOOK, E * cap, 4}, {EJ_F_KEY, 2, 4},
    };
    uint64_t off = 0;
    for (auto& f : fields) {
        L_.off[f.f] = off;
        L_.count[f.f] = f.n;
        L_.esz[f.f] = f.esz;
        off = align256(off + f.n * f.esz);
    }
    L_.sizes.n_actions = nA;
    L_.sizes.obs_dim = D;
    L_.sizes.gobs_dim = G;
    L_.sizes.mask_words = W;
    L_.sizes.levels = L;
    L_.sizes.book_cap = cap;
    L_.sizes.threads = NT;
    L_.sizes.smem_bytes = (int32_t)sl.total;
    L_.sizes.state_bytes = off;
    if (lay) *lay = L_;

    if (kp) {
        KParams k;
        memset(&k, 0, sizeof k);
        k.E = p->E; k.e0 = 0; k.ne = p->E; k.A = p->A; k.A_s = A_s; k.R = p->R; k.P = p->P; k.nb = p->nb; k.L = L;
        k.nA = nA; k.D = D; k.G = G; k.W = W; k.M = M; k.cap = cap;
        k.T_ep = p->T_ep; k.T_tax = p->T_tax; k.expire = p->expire; k.max_orders = p->max_orders;
        k.Rk = p->Rk; k.Rd = p->Rd; k.allow_noop = p->allow_noop != 0; k.gov_enabled = p->gov_enabled != 0;
        k.tax_levels = p->tax_levels;
        k.start_coin = p->start_coin; k.ome = 1.0f - p->eta; k.omega = p->omega;
        k.lg = p->labor_gather; k.lc = p->labor_craft; k.lt = p->labor_trade;
        k.craft_coin = p->craft_coin; k.gather_rho = p->gather_rho; k.tick = p->price_tick;
        k.skill_gain = p->skill_gain; k.skill_max = p->skill_max; k.skill_init = p->skill_init;
        for (int q = 0; q < p->P; ++q) {
            k.ticks[q] = p->price_ticks[q];
            volatile float prod = p->price_tick * (float)p->price_ticks[q];   // one float rounding
            k.price[q] = prod;
        }
        for (int b = 0; b + 1 < p->nb; ++b) k.th[b] = p->thresholds[b];
        *kp = k;
    }
    return EJ_OK;
}

DevState state_pointers(const Layout& lay, void* base) {
    char* b = (char*)base;
    DevState s;
    s.coin = (float*)(b + lay.off[EJ_F_COIN]);
    s.esc = (int*)(b + lay.off[EJ_F_ESC]);
    s.income = (float*)(b + lay.off[EJ_F_INCOME]);
    s.uprev = (float*)(b + lay.off[EJ_F_UPREV]);
    s.nord = (int*)(b + lay.off[EJ_F_NORD]);
    s.counts = (int*)(b + lay.off[EJ_F_COUNTS]);
    s.sc = (float*)(b + lay.off[EJ_F_SC]);
    s.inv = (int*)(b + lay.off[EJ_F_INV]);
    s.inve = (int*)(b + lay.off[EJ_F_INVE]);
    s.sg = (float*)(b + lay.off[EJ_F_SG]);
    s.t = (int*)(b + lay.off[EJ_F_T]);
    s.gstep = (uint32_t*)(b + lay.off[EJ_F_GSTEP]);
    s.episode = (uint32_t*)(b + lay.off[EJ_F_EPISODE]);
    s.pop = (int*)(b + lay.off[EJ_F_POP]);
    s.rates = (float*)(b + lay.off[EJ_F_RATES]);
    s.ugprev = (float*)(b + lay.off[EJ_F_UGPREV]);
    s.lvl = (int*)(b + lay.off[EJ_F_LEVEL_COUNT]);
    s.book = (uint32_t*)(b + lay.off[EJ_F_BOOK]);
    s.key = (uint32_t*)(b + lay.off[EJ_F_KEY]);
    return s;
}

}  // namespace ej

using namespace ej;

extern "C" {

const char* ej_last_error(void) { return g_err; }

ej_status ej_params_default(EjParams* p) {
    if (!p) return fail(EJ_ERR_ARG, "params is NULL");
    memset(p, 0, sizeof *p);
    p->E = 1; p->A = 100; p->R = 2; p->P = 5; p->nb = 3;
    p->T_ep = 1000; p->T_tax = 100; p->expire = 30; p->max_orders = 15;
    p->Rk = 2; p->Rd = 2; p->allow_noop = 1; p->gov_enabled = 1; p->tax_levels = 21;
    p->start_coin = 15.0f; p->eta = 0.27f; p->omega = 1.0f;
    p->labor_gather = 1.0f; p->labor_craft = 1.0f; p->labor_trade = 0.05f;
    p->craft_coin = 10.0f; p->gather_rho = 1.1f; p->price_tick = 2.0f;
    for (int q = 0; q < 5; ++q) p->price_ticks[q] = q + 1;
    p->thresholds[0] = 50.0f; p->thresholds[1] = 100.0f;
    p->skill_gain = 0.0f; p->skill_max = 5.0f; p->skill_init = 0;
    return EJ_OK;
}

ej_status ej_sizes(const EjParams* p, EjSizes* s) {
    Layout lay;
    ej_status st = derive(p, &lay, nullptr);
    if (st != EJ_OK) return st;
    if (s) *s = lay.sizes;
    return EJ_OK;
}

ej_status ej_state_field(const EjParams* p, int32_t field, uint64_t* offset, uint64_t* count,
                         int32_t* elem_bytes) {
    Layout lay;
    ej_status st = derive(p, &lay, nullptr);
    if (st != EJ_OK) return st;
    if (field < 0 || field >= EJ_F_COUNT_) return fail(EJ_ERR_ARG, "unknown field %d", field);
    if (offset) *offset = lay.off[field];
    if (count) *count = lay.count[field];
    if (elem_bytes) *elem_bytes = lay.esz[field];
    return EJ_OK;
}

ej_status env_reset(const EjParams* p, void* state, const int32_t* pop_sizes, uint64_t seed,
                    float* obs, float* gobs, uint32_t* mask, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    if (!state) return fail(EJ_ERR_ARG, "state is NULL");
    if ((uintptr_t)state % 256) return fail(EJ_ERR_ARG, "state must be 256-byte aligned");
    DevIO io;
    memset(&io, 0, sizeof io);
    io.obs = obs; io.gobs = gobs; io.mask = mask; io.pop_sizes = pop_sizes;
    return launch_env(kp, lay, state_pointers(lay, state), io, 0, MODE_RESET, seed, (cudaStream_t)stream);
}

ej_status env_step(const EjParams* p, void* state, int32_t n_steps, const int32_t* act,
                   const int32_t* gov_act, const float* gather_u, const uint32_t* tb,
                   float* rew, float* grew, uint8_t* done, float* obs, float* gobs,
                   uint32_t* mask, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    if (!state) return fail(EJ_ERR_ARG, "state is NULL");
    if ((uintptr_t)state % 256) return fail(EJ_ERR_ARG, "state must be 256-byte aligned");
    if (n_steps < 0) return fail(EJ_ERR_ARG, "n_steps must be >= 0");
    if ((gather_u == nullptr) != (tb == nullptr))
        return fail(EJ_ERR_ARG, "gather_u and tb must be both given or both NULL");
    if (!act && gather_u) return fail(EJ_ERR_ARG, "gather_u and tb need act");
    if (n_steps == 0) return EJ_OK;
    DevIO io;
    memset(&io, 0, sizeof io);
    io.act = act; io.gov_act = gov_act; io.gather_u = gather_u; io.tb = tb;
    io.rew = rew; io.grew = grew; io.done = done; io.obs = obs; io.gobs = gobs; io.mask = mask;
    int mode = (act ? 0 : MODE_POP_DRAW) | (gather_u ? 0 : MODE_AUX_DRAW) | (gov_act ? 0 : MODE_GOV_DRAW);
    return launch_env(kp, lay, state_pointers(lay, state), io, n_steps, mode, 0, (cudaStream_t)stream);
}

ej_status ej_fill_draws(const EjParams* p, uint64_t seed, uint32_t g0, int32_t n_steps,
                        int32_t* act, float* gather_u, uint32_t* tb, float* policy_u,
                        int32_t* gov_act, void* stream) {
    Layout lay;
    KParams kp;
    ej_status st = derive(p, &lay, &kp);
    if (st != EJ_OK) return st;
    if (n_steps < 0) return fail(EJ_ERR_ARG, "n_steps must be >= 0");
    if (n_steps == 0) return EJ_OK;
    return launch_fill_draws(kp, seed, g0, n_steps, act, gather_u, tb, policy_u, gov_act,
                             (cudaStream_t)stream);
}

}  // extern "C"
