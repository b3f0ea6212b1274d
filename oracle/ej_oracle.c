/*
 * CPU oracle of the EconoJax environment (arxiv 2410.22165, Section 3).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline leg of bench.py; never by the product path.  Build with
 *   gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (no FMA contraction: every float operation below rounds once, in the
 * order written).
 *
 * The step applies the rules in this order (readings of the paper where it
 * is silent are marked READING):
 *   0. period start: the government's rates take effect        (Sec. 3, "Setting tax rates")
 *   1. population actions, each agent on its own state          (Sec. 3, "Population Agents")
 *      - invalid (masked) actions act as NO-OP with no labor     (Sec. 3, "Action masking")
 *      - gather: floor(SG + rho), rho = gather_rho * u           (Sec. 3, "Collecting resources")
 *      - craft: R_d richest resources, R_k units each            (Sec. 3, "Crafting")
 *      - buy/sell one unit at a price level, into escrow         (Sec. 3, "Trading")
 *   2. matching per resource: best bids against best asks,
 *      ties by age then by a random key; price of the later order (Sec. 3 "Trading"; App. A)
 *   3. expiry of orders that took part in `expire` rounds        (Sec. 3 "Trading"; Table 2)
 *   4. period end: bracket tax on period earnings, uniform
 *      redistribution                                            (Sec. 3, "Setting tax rates")
 *   5. rewards: change in isoelastic utility (Eq. 1, Eq. 2) and
 *      in social welfare (Eq. 3-5)                               (Sec. 3, "Government Agent")
 *   6. end of episode: restart with new skills (functional reset) (Sec. 3, "Overall design")
 *   7. observation and action mask of the new state              (Sec. 3; App. A)
 *
 * Parity pins (tests/test_oracle_*.py): the worked tax example of Section 3
 * (130 coin of earnings under rates 10/30/50 % and brackets [50;100] pays 35);
 * the action counts of Section 5 (30 actions at r=4, 86 at r=12 with three
 * prices); hand-enumerated markets; conservation of coin and resources through
 * escrow; brute-force gini; the gather formula at its boundaries.
 * Whole-episode trajectories are "parity unpinned" against the paper (it
 * prints none).
 */
#include "ej_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int side;      /* 0 = buy (bid), 1 = sell (ask) */
    int r;         /* resource */
    int p;         /* price level */
    int agent;
    int step;      /* step at which the order was placed (its age) */
    uint32_t tb;   /* random tie-break key drawn when the order was placed */
    int alive;
} order_t;

struct orc_env {
    orc_params prm;
    int A;
    int t;          /* step within the episode */
    int episode;
    float rates32[ORC_MAX_NB];
    double rates64[ORC_MAX_NB];
    double ug_prev;           /* government utility after the previous step */
    /* per agent */
    float* coin32;            /* liquid coin, decision mirror (float) */
    double* coin64;           /* liquid coin, reported track (double) */
    float* income32;          /* earnings in the current tax period, mirror */
    double* income64;         /* earnings in the current tax period, reported */
    int* esc_ticks;           /* coin in escrow, in price ticks */
    int* inv;                 /* [A*R] liquid resources */
    int* inv_esc;             /* [A*R] resources in escrow */
    int* n_orders;            /* active orders */
    int* n_gather;            /* actions performed this episode (labor accounting) */
    int* n_craft;
    int* n_trade;
    float* sg;                /* [A*R] gather skill */
    float* sc;                /* craft skill */
    double* u_prev;           /* utility after the previous step */
    /* market */
    order_t* book;
    int n_book, cap_book;
    int trades[ORC_MAX_R];
    int64_t tick_volume[ORC_MAX_R];
};

/* ------------------------------------------------------------------ sizes */

/* Action layout (READING; pinned by Section 5: 30 actions at r=4 and 86 at
 * r=12 with three prices and NO-OP):
 *   0 NO-OP | 1..R gather r | R+1 craft | R+2+r*P+p buy r at level p |
 *   R+2+R*P+r*P+p sell r at level p.                                     */
int orc_num_actions(const orc_params* p) { return 2 + p->R + 2 * p->R * p->P; }

/* Population observation (READING of Fig. 1, which is not available):
 * coin, coin in escrow, labor, inv[R], inv_esc[R], SG[R], SC,
 * orders/max_orders, per resource {best bid, best ask, #bids/A, #asks/A},
 * rates[nb], period earnings, fraction of the tax period left, t/T_ep.      */
int orc_obs_dim(const orc_params* p) { return 8 + 7 * p->R + p->nb; }

/* Government observation (READING of Fig. 1 / App. A: statistics, not
 * individual states): mean, std, median of {total coin, period earnings,
 * labor}, then rates[nb], fraction of the tax period left, t/T_ep.         */
int orc_gobs_dim(const orc_params* p) { return 3 * 3 + p->nb + 2; }

int orc_mask_words(const orc_params* p) { return (orc_num_actions(p) + 31) / 32; }

/* ------------------------------------------------------- closed forms */

/* Eq. 1: isoelastic utility of coin minus labor. */
double orc_isoelastic(double coin, double labor, double eta) {
    return (pow(coin, 1.0 - eta) - 1.0) / (1.0 - eta) - labor;
}

/* Gini index (Section 3, "Government Agent"): mean absolute difference over
 * all ordered pairs divided by twice the mean, written out as the double sum.
 * Zero when everybody holds nothing. */
double orc_gini(const double* x, int n) {
    double total = 0.0, pair_sum = 0.0;
    for (int i = 0; i < n; ++i) total += x[i];
    if (n == 0 || total <= 0.0) return 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) pair_sum += fabs(x[i] - x[j]);
    return pair_sum / (2.0 * (double)n * total);
}

/* Section 3, "Setting tax rates": marginal tax over brackets
 * [0, th0), [th0, th1), ..., [th_{nb-2}, inf). */
double orc_bracket_tax(double income, const double* rates, const double* th, int nb) {
    double tax = 0.0;
    for (int b = 0; b < nb; ++b) {
        double lo = (b == 0) ? 0.0 : th[b - 1];
        double hi = (b == nb - 1) ? INFINITY : th[b];
        double part = income - lo;
        if (part < 0.0) part = 0.0;
        if (part > hi - lo) part = hi - lo;
        tax += rates[b] * part;
    }
    return tax;
}

/* Float mirror of the bracket tax: the same sum, one rounding per operation,
 * brackets in ascending order. */
static float bracket_tax32(float income, const float* rates, const double* th, int nb) {
    float tax = 0.0f;
    for (int b = 0; b < nb; ++b) {
        float lo = (b == 0) ? 0.0f : (float)th[b - 1];
        float part = income - lo;
        if (part < 0.0f) part = 0.0f;
        if (b < nb - 1) {
            float width = (float)th[b] - lo;
            if (part > width) part = width;
        }
        float term = rates[b] * part;
        tax = tax + term;
    }
    return tax;
}

/* Float mirror of the tax pool (READING R15; the paper fixes no order of
 * summation): the agents in blocks of 32 in agent order, zero-padded; within
 * a block a butterfly sum, which at offsets 16, 8, 4, 2, 1 replaces every
 * entry t[j] by t[j] + t[j ^ offset] (each addition rounded once), the block
 * sum being entry 0 at the end; the block sums added one after another in
 * agent order, starting from 0. */
static float pool_sum32(const float* tax, int A) {
    float pool = 0.0f;
    for (int b0 = 0; b0 < A; b0 += 32) {
        float t[32], u[32];
        for (int j = 0; j < 32; ++j) t[j] = (b0 + j < A) ? tax[b0 + j] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) {
            for (int j = 0; j < 32; ++j) u[j] = t[j] + t[j ^ o];
            memcpy(t, u, sizeof t);
        }
        pool = pool + t[0];
    }
    return pool;
}

/* --------------------------------------------------------- life cycle */

orc_env* orc_env_new(const orc_params* p, int A) {
    orc_env* env = (orc_env*)calloc(1, sizeof(orc_env));
    env->prm = *p;
    env->A = A;
    int R = p->R;
    env->coin32 = (float*)calloc(A, sizeof(float));
    env->coin64 = (double*)calloc(A, sizeof(double));
    env->income32 = (float*)calloc(A, sizeof(float));
    env->income64 = (double*)calloc(A, sizeof(double));
    env->esc_ticks = (int*)calloc(A, sizeof(int));
    env->inv = (int*)calloc((size_t)A * R, sizeof(int));
    env->inv_esc = (int*)calloc((size_t)A * R, sizeof(int));
    env->n_orders = (int*)calloc(A, sizeof(int));
    env->n_gather = (int*)calloc(A, sizeof(int));
    env->n_craft = (int*)calloc(A, sizeof(int));
    env->n_trade = (int*)calloc(A, sizeof(int));
    env->sg = (float*)calloc((size_t)A * R, sizeof(float));
    env->sc = (float*)calloc(A, sizeof(float));
    env->u_prev = (double*)calloc(A, sizeof(double));
    env->cap_book = A * (p->max_orders + 1) + 16;
    env->book = (order_t*)calloc(env->cap_book, sizeof(order_t));
    return env;
}

void orc_env_free(orc_env* env) {
    if (!env) return;
    free(env->coin32); free(env->coin64); free(env->income32); free(env->income64);
    free(env->esc_ticks); free(env->inv); free(env->inv_esc); free(env->n_orders);
    free(env->n_gather); free(env->n_craft); free(env->n_trade);
    free(env->sg); free(env->sc); free(env->u_prev); free(env->book);
    free(env);
}

static double labor_of(const orc_env* env, int i) {
    const orc_params* p = &env->prm;
    return p->labor_gather * env->n_gather[i] + p->labor_craft * env->n_craft[i]
         + p->labor_trade * env->n_trade[i];
}

static double total_coin64(const orc_env* env, int i) {
    return env->coin64[i] + env->prm.price_tick * env->esc_ticks[i];
}

/* Social welfare of Eq. 3-5 on total coin (READING of the garbled Eq. 4:
 * Eq = omega * (1 - gini) + (1 - omega)). */
static double gov_utility(const orc_env* env) {
    int A = env->A;
    double* c = (double*)malloc(sizeof(double) * (A > 0 ? A : 1));
    double prod = 0.0;
    for (int i = 0; i < A; ++i) { c[i] = total_coin64(env, i); prod += c[i]; }
    double eq = env->prm.omega * (1.0 - orc_gini(c, A)) + (1.0 - env->prm.omega);
    free(c);
    return eq * prod;
}

/* Start of an episode (Section 3: skills are set at initialization and stay
 * fixed through the episode; Table 2: starting coin 15). */
static void start_episode(orc_env* env, const float* sg, const float* sc) {
    const orc_params* p = &env->prm;
    int A = env->A, R = p->R;
    env->t = 0;
    for (int b = 0; b < ORC_MAX_NB; ++b) { env->rates32[b] = 0.0f; env->rates64[b] = 0.0; }
    for (int i = 0; i < A; ++i) {
        env->coin32[i] = (float)p->start_coin;
        env->coin64[i] = (double)(float)p->start_coin;
        env->income32[i] = 0.0f;
        env->income64[i] = 0.0;
        env->esc_ticks[i] = 0;
        env->n_orders[i] = 0;
        env->n_gather[i] = env->n_craft[i] = env->n_trade[i] = 0;
        for (int r = 0; r < R; ++r) {
            env->inv[i * R + r] = 0;
            env->inv_esc[i * R + r] = 0;
            env->sg[i * R + r] = sg[i * R + r];
        }
        env->sc[i] = sc[i];
        env->u_prev[i] = orc_isoelastic(total_coin64(env, i), 0.0, p->eta);
    }
    env->n_book = 0;
    for (int r = 0; r < ORC_MAX_R; ++r) { env->trades[r] = 0; env->tick_volume[r] = 0; }
    env->ug_prev = gov_utility(env);
}

void orc_env_reset(orc_env* env, const float* sg, const float* sc) {
    env->episode = 0;
    start_episode(env, sg, sc);
}

/* --------------------------------------------------------------- masks */

static float price32(const orc_params* p, int level) {
    return (float)p->price_tick * (float)p->price_ticks[level];
}

/* Section 5: the skill after a gather or craft.  The relative bonus is
 * skill_gain at skill 0 and falls linearly to 0 at skill_max (READING of the
 * section's half-percent bonus that vanishes at the skill ceiling of 5);
 * float32, every operation rounded once. */
static float skill_up(const orc_params* p, float s) {
    if (!(p->skill_gain > 0.0)) return s;
    const float smax = (float)p->skill_max;
    const float room = 1.0f - s / smax;
    const float gain = (float)p->skill_gain * room;
    const float up = s + s * gain;
    return up < smax ? up : smax;
}

/* Section 3, "Crafting": can the agent craft?  It needs R_k units of each of
 * R_d different resources. */
static int can_craft(const orc_env* env, int i) {
    const orc_params* p = &env->prm;
    int enough = 0;
    for (int r = 0; r < p->R; ++r) enough += env->inv[i * p->R + r] >= p->Rk;
    return enough >= p->Rd;
}

/* Section 3, "Action masking": is action a available to agent i now? */
static int action_valid(const orc_env* env, int i, int a) {
    const orc_params* p = &env->prm;
    int R = p->R, P = p->P;
    if (a < 0 || a >= orc_num_actions(p)) return 0;
    if (a == 0) return p->allow_noop != 0;
    if (a <= R) return 1;                              /* gather */
    if (a == R + 1) return can_craft(env, i);          /* craft */
    int j = a - (R + 2);
    if (j < R * P) {                                   /* buy: needs the price in liquid coin */
        int level = j % P;
        return env->n_orders[i] < p->max_orders && env->coin32[i] >= price32(p, level);
    }
    j -= R * P;                                        /* sell: needs one unit */
    int r = j / P;
    return env->n_orders[i] < p->max_orders && env->inv[i * R + r] >= 1;
}

/* ------------------------------------------------------------- market */

static int cmp_bids(const void* x, const void* y) {
    const order_t* a = *(const order_t* const*)x;
    const order_t* b = *(const order_t* const*)y;
    if (a->p != b->p) return a->p > b->p ? -1 : 1;          /* high bids first */
    if (a->step != b->step) return a->step < b->step ? -1 : 1;  /* then older */
    if (a->tb != b->tb) return a->tb < b->tb ? -1 : 1;      /* then by the random key */
    return a->agent < b->agent ? -1 : (a->agent > b->agent);
}

static int cmp_asks(const void* x, const void* y) {
    const order_t* a = *(const order_t* const*)x;
    const order_t* b = *(const order_t* const*)y;
    if (a->p != b->p) return a->p < b->p ? -1 : 1;          /* low asks first */
    if (a->step != b->step) return a->step < b->step ? -1 : 1;
    if (a->tb != b->tb) return a->tb < b->tb ? -1 : 1;
    return a->agent < b->agent ? -1 : (a->agent > b->agent);
}

/* Coin and income changes of the market are counted in whole price ticks
 * during the step and added to the float tracks once at the end. */
typedef struct { int64_t coin_ticks, income_ticks; } tick_delta;

/* Section 3, "Trading" and Appendix A: sort bids high-to-low and asks
 * low-to-high (ties: older first, then the random key), pair the k-th bid
 * with the k-th ask while the bid is at least the ask.  The trade happens at
 * the price of the newer of the two orders (READING: the ask's price when both were
 * placed in the same step). */
static void match_resource(orc_env* env, int r, tick_delta* d) {
    const orc_params* p = &env->prm;
    int R = p->R;
    order_t** bids = (order_t**)malloc(sizeof(order_t*) * (env->n_book + 1));
    order_t** asks = (order_t**)malloc(sizeof(order_t*) * (env->n_book + 1));
    int nbid = 0, nask = 0;
    for (int k = 0; k < env->n_book; ++k) {
        order_t* o = &env->book[k];
        if (!o->alive || o->r != r) continue;
        if (o->side == 0) bids[nbid++] = o; else asks[nask++] = o;
    }
    qsort(bids, nbid, sizeof(order_t*), cmp_bids);
    qsort(asks, nask, sizeof(order_t*), cmp_asks);
    for (int k = 0; k < nbid && k < nask; ++k) {
        order_t* b = bids[k];
        order_t* s = asks[k];
        if (b->p < s->p) break;                 /* bid below ask: no more trades */
        int bid_ticks = p->price_ticks[b->p];
        int trade_ticks = (b->step > s->step) ? bid_ticks : p->price_ticks[s->p];
        /* buyer: pays the trade price out of escrow, gets the rest back */
        env->esc_ticks[b->agent] -= bid_ticks;
        d[b->agent].coin_ticks += bid_ticks - trade_ticks;
        env->inv[b->agent * R + r] += 1;
        env->n_orders[b->agent] -= 1;
        /* seller: the unit leaves escrow, the price is earned */
        env->inv_esc[s->agent * R + r] -= 1;
        d[s->agent].coin_ticks += trade_ticks;
        d[s->agent].income_ticks += trade_ticks;
        env->n_orders[s->agent] -= 1;
        b->alive = 0;
        s->alive = 0;
        env->trades[r] += 1;
        env->tick_volume[r] += trade_ticks;
    }
    free(bids);
    free(asks);
}

/* Table 2 ("trade order expire time 30"): an order takes part in `expire`
 * matching rounds, its own step's included, and then leaves the market; the
 * escrowed coin or unit goes back to its owner (READING: the paper gives
 * orders a limited lifetime measured in steps, not how the boundary step
 * counts). */
static void expire_orders(orc_env* env, tick_delta* d) {
    const orc_params* p = &env->prm;
    int R = p->R;
    for (int k = 0; k < env->n_book; ++k) {
        order_t* o = &env->book[k];
        if (!o->alive) continue;
        if (env->t - o->step + 1 < p->expire) continue;
        if (o->side == 0) {
            int ticks = p->price_ticks[o->p];
            env->esc_ticks[o->agent] -= ticks;
            d[o->agent].coin_ticks += ticks;
        } else {
            env->inv_esc[o->agent * R + o->r] -= 1;
            env->inv[o->agent * R + o->r] += 1;
        }
        env->n_orders[o->agent] -= 1;
        o->alive = 0;
    }
    int w = 0;
    for (int k = 0; k < env->n_book; ++k)
        if (env->book[k].alive) env->book[w++] = env->book[k];
    env->n_book = w;
}

/* --------------------------------------------------------- observation */

static int cmp_double(const void* x, const void* y) {
    double a = *(const double*)x, b = *(const double*)y;
    return (a > b) - (a < b);
}

static void stats3(const double* x, int n, double* out) {
    double mean = 0.0, var = 0.0;
    for (int i = 0; i < n; ++i) mean += x[i];
    mean /= (n > 0 ? n : 1);
    for (int i = 0; i < n; ++i) var += (x[i] - mean) * (x[i] - mean);
    var /= (n > 0 ? n : 1);
    double* s = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
    memcpy(s, x, sizeof(double) * n);
    qsort(s, n, sizeof(double), cmp_double);
    double median = 0.0;
    if (n > 0) median = (n % 2) ? s[n / 2] : 0.5 * (s[n / 2 - 1] + s[n / 2]);
    free(s);
    out[0] = mean;
    out[1] = sqrt(var);
    out[2] = median;
}

void orc_env_observe(const orc_env* env, double* obs, double* gobs, uint32_t* mask) {
    const orc_params* p = &env->prm;
    int A = env->A, R = p->R, P = p->P, nb = p->nb;
    int D = orc_obs_dim(p), W = orc_mask_words(p), nA = orc_num_actions(p);
    double period_left = (double)(p->T_tax - env->t % p->T_tax) / (double)p->T_tax;
    double time_frac = (double)env->t / (double)p->T_ep;
    /* market statistics (App. A: highest / lowest / number of orders) */
    double best_bid[ORC_MAX_R], best_ask[ORC_MAX_R], n_bid[ORC_MAX_R], n_ask[ORC_MAX_R];
    for (int r = 0; r < R; ++r) {
        int hi = -1, lo = P, cb = 0, ca = 0;
        for (int k = 0; k < env->n_book; ++k) {
            const order_t* o = &env->book[k];
            if (o->r != r) continue;
            if (o->side == 0) { cb++; if (o->p > hi) hi = o->p; }
            else { ca++; if (o->p < lo) lo = o->p; }
        }
        best_bid[r] = hi >= 0 ? p->price_tick * p->price_ticks[hi] : 0.0;
        best_ask[r] = lo < P ? p->price_tick * p->price_ticks[lo] : 0.0;
        n_bid[r] = (double)cb / (double)A;
        n_ask[r] = (double)ca / (double)A;
    }
    if (obs) {
        for (int i = 0; i < A; ++i) {
            double* o = obs + (size_t)i * D;
            int k = 0;
            o[k++] = env->coin64[i];
            o[k++] = p->price_tick * env->esc_ticks[i];
            o[k++] = labor_of(env, i);
            for (int r = 0; r < R; ++r) o[k++] = env->inv[i * R + r];
            for (int r = 0; r < R; ++r) o[k++] = env->inv_esc[i * R + r];
            for (int r = 0; r < R; ++r) o[k++] = env->sg[i * R + r];
            o[k++] = env->sc[i];
            o[k++] = (double)env->n_orders[i] / (double)p->max_orders;
            for (int r = 0; r < R; ++r) {
                o[k++] = best_bid[r];
                o[k++] = best_ask[r];
                o[k++] = n_bid[r];
                o[k++] = n_ask[r];
            }
            for (int b = 0; b < nb; ++b) o[k++] = env->rates64[b];
            o[k++] = env->income64[i];
            o[k++] = period_left;
            o[k++] = time_frac;
        }
    }
    if (gobs) {
        int M = 3;
        double* x = (double*)malloc(sizeof(double) * (A > 0 ? A : 1));
        for (int m = 0; m < M; ++m) {
            for (int i = 0; i < A; ++i) {
                if (m == 0) x[i] = total_coin64(env, i);
                else if (m == 1) x[i] = env->income64[i];
                else x[i] = labor_of(env, i);
            }
            stats3(x, A, gobs + 3 * m);
        }
        free(x);
        int k = 3 * M;
        for (int b = 0; b < nb; ++b) gobs[k++] = env->rates64[b];
        gobs[k++] = period_left;
        gobs[k++] = time_frac;
    }
    if (mask) {
        for (int i = 0; i < A; ++i) {
            for (int w = 0; w < W; ++w) mask[(size_t)i * W + w] = 0u;
            for (int a = 0; a < nA; ++a)
                if (action_valid(env, i, a)) mask[(size_t)i * W + a / 32] |= 1u << (a % 32);
        }
    }
}

/* ----------------------------------------------------------------- step */

void orc_env_step(orc_env* env, const int32_t* act, const int32_t* gov_act,
                  const float* gather_u, const uint32_t* tb,
                  const float* next_sg, const float* next_sc,
                  double* rew, double* grew, int32_t* done,
                  double* obs, double* gobs, uint32_t* mask) {
    const orc_params* p = &env->prm;
    int A = env->A, R = p->R, P = p->P, nb = p->nb;
    int t = env->t;
    for (int r = 0; r < R; ++r) { env->trades[r] = 0; env->tick_volume[r] = 0; }

    /* 0. Period start: the government sets the rates of the coming period,
     *    one of tax_levels equally spaced levels from 0 to 100 % per bracket. */
    if (p->gov_enabled && t % p->T_tax == 0) {
        for (int b = 0; b < nb; ++b) {
            int level = gov_act[b];
            if (level < 0) level = 0;
            if (level > p->tax_levels - 1) level = p->tax_levels - 1;
            env->rates32[b] = (float)level / (float)(p->tax_levels - 1);
            env->rates64[b] = (double)level / (double)(p->tax_levels - 1);
        }
    }

    /* 1. Population actions.  Validity is judged on the agent's state at the
     *    start of the step; an invalid action does nothing. */
    for (int i = 0; i < A; ++i) {
        int a = act[i];
        if (!action_valid(env, i, a) || a == 0) continue;
        if (a <= R) {                                         /* gather resource a-1 */
            int r = a - 1;
            float rho = (float)p->gather_rho * gather_u[i];
            float s = env->sg[i * R + r] + rho;
            env->inv[i * R + r] += (int)floorf(s);
            env->n_gather[i] += 1;
            env->sg[i * R + r] = skill_up(p, env->sg[i * R + r]);
        } else if (a == R + 1) {                              /* craft */
            int used[ORC_MAX_R] = {0};
            for (int k = 0; k < p->Rd; ++k) {                 /* richest first, lower index on ties */
                int best = -1;
                for (int r = 0; r < R; ++r)
                    if (!used[r] && (best < 0 || env->inv[i * R + r] > env->inv[i * R + best])) best = r;
                used[best] = 1;
                env->inv[i * R + best] -= p->Rk;
            }
            float gain32 = env->sc[i] * (float)p->craft_coin;
            env->coin32[i] = env->coin32[i] + gain32;
            env->income32[i] = env->income32[i] + gain32;
            double gain64 = (double)env->sc[i] * p->craft_coin;
            env->coin64[i] += gain64;
            env->income64[i] += gain64;
            env->n_craft[i] += 1;
            env->sc[i] = skill_up(p, env->sc[i]);
        } else {                                              /* place one order */
            int j = a - (R + 2);
            int side = j >= R * P;
            if (side) j -= R * P;
            int r = j / P, level = j % P;
            if (side == 0) {                                  /* buy: price into escrow */
                env->coin32[i] = env->coin32[i] - price32(p, level);
                env->coin64[i] -= p->price_tick * p->price_ticks[level];
                env->esc_ticks[i] += p->price_ticks[level];
            } else {                                          /* sell: one unit into escrow */
                env->inv[i * R + r] -= 1;
                env->inv_esc[i * R + r] += 1;
            }
            order_t* o = &env->book[env->n_book++];
            o->side = side; o->r = r; o->p = level; o->agent = i;
            o->step = t; o->tb = tb[i]; o->alive = 1;
            env->n_orders[i] += 1;
            env->n_trade[i] += 1;
        }
    }

    /* 2-3. Market: match every resource, then expire old orders. */
    tick_delta* d = (tick_delta*)calloc(A > 0 ? A : 1, sizeof(tick_delta));
    for (int r = 0; r < R; ++r) match_resource(env, r, d);
    expire_orders(env, d);
    for (int i = 0; i < A; ++i) {
        float coin_add = (float)p->price_tick * (float)d[i].coin_ticks;
        float inc_add = (float)p->price_tick * (float)d[i].income_ticks;
        env->coin32[i] = env->coin32[i] + coin_add;
        env->income32[i] = env->income32[i] + inc_add;
        env->coin64[i] += p->price_tick * (double)d[i].coin_ticks;
        env->income64[i] += p->price_tick * (double)d[i].income_ticks;
    }
    free(d);

    /* 4. Period end: tax the period's earnings bracket by bracket (capped at
     *    the liquid coin the agent holds), pay the total back in equal
     *    shares, start a new period of earnings. */
    if ((t + 1) % p->T_tax == 0) {
        if (p->gov_enabled) {
            float* tax32 = (float*)malloc(sizeof(float) * (A > 0 ? A : 1));
            double* tax64 = (double*)malloc(sizeof(double) * (A > 0 ? A : 1));
            double pool64 = 0.0;
            for (int i = 0; i < A; ++i) {
                tax32[i] = bracket_tax32(env->income32[i], env->rates32, p->thresholds, nb);
                if (tax32[i] > env->coin32[i]) tax32[i] = env->coin32[i];
                tax64[i] = orc_bracket_tax(env->income64[i], env->rates64, p->thresholds, nb);
                if (tax64[i] > env->coin64[i]) tax64[i] = env->coin64[i];
                pool64 += tax64[i];
            }
            float pool32 = pool_sum32(tax32, A);
            float share32 = pool32 / (float)A;
            double share64 = pool64 / (double)A;
            for (int i = 0; i < A; ++i) {
                float after = env->coin32[i] - tax32[i];
                env->coin32[i] = after + share32;
                env->coin64[i] = env->coin64[i] - tax64[i] + share64;
            }
            free(tax32);
            free(tax64);
        }
        for (int i = 0; i < A; ++i) { env->income32[i] = 0.0f; env->income64[i] = 0.0; }
    }

    /* 5. Rewards: Eq. 2 on the utility of Eq. 1 (coin counts escrow, READING)
     *    and the same difference on the social welfare of Eq. 3. */
    for (int i = 0; i < A; ++i) {
        double u = orc_isoelastic(total_coin64(env, i), labor_of(env, i), p->eta);
        if (rew) rew[i] = u - env->u_prev[i];
        env->u_prev[i] = u;
    }
    double ug = gov_utility(env);
    if (grew) *grew = ug - env->ug_prev;
    env->ug_prev = ug;

    /* 6. End of episode: functional reset with the next episode's skills. */
    env->t = t + 1;
    int ended = env->t == p->T_ep;
    if (done) *done = ended;
    if (ended) {
        env->episode += 1;
        start_episode(env, next_sg, next_sc);
    }

    /* 7. Observation of the new state. */
    orc_env_observe(env, obs, gobs, mask);
}

void orc_env_run(orc_env* env, int n, const int32_t* act, const int32_t* gov_act,
                 const float* gather_u, const uint32_t* tb,
                 const float* later_sg, const float* later_sc,
                 double* rew, double* grew, int32_t* done,
                 double* obs, double* gobs, uint32_t* mask) {
    const orc_params* p = &env->prm;
    int A = env->A, R = p->R;
    int D = orc_obs_dim(p), G = orc_gobs_dim(p), W = orc_mask_words(p);
    int ep0 = env->episode;
    for (int s = 0; s < n; ++s) {
        int k = env->episode - ep0;   /* episodes started during this run so far */
        const float* nsg = later_sg ? later_sg + (size_t)k * A * R : NULL;
        const float* nsc = later_sc ? later_sc + (size_t)k * A : NULL;
        orc_env_step(env, act + (size_t)s * A, gov_act + (size_t)s * p->nb,
                     gather_u + (size_t)s * A, tb + (size_t)s * A, nsg, nsc,
                     rew ? rew + (size_t)s * A : NULL, grew ? grew + s : NULL,
                     done ? done + s : NULL, obs ? obs + (size_t)s * A * D : NULL,
                     gobs ? gobs + (size_t)s * G : NULL,
                     mask ? mask + (size_t)s * A * W : NULL);
    }
}

/* ------------------------------------------------------------ read-out */

void orc_env_get_info(const orc_env* env, orc_env_info* info) {
    info->t = env->t;
    info->episode = env->episode;
    info->n_book = env->n_book;
    for (int b = 0; b < ORC_MAX_NB; ++b) {
        info->rates32[b] = env->rates32[b];
        info->rates64[b] = env->rates64[b];
    }
    info->ug_prev = env->ug_prev;
}

void orc_env_get_agents(const orc_env* env, float* coin32, double* coin64,
                        float* income32, double* income64, int32_t* esc_ticks,
                        int32_t* inv, int32_t* inv_esc, int32_t* n_orders,
                        int32_t* counts, double* u_prev) {
    int A = env->A, R = env->prm.R;
    for (int i = 0; i < A; ++i) {
        if (coin32) coin32[i] = env->coin32[i];
        if (coin64) coin64[i] = env->coin64[i];
        if (income32) income32[i] = env->income32[i];
        if (income64) income64[i] = env->income64[i];
        if (esc_ticks) esc_ticks[i] = env->esc_ticks[i];
        if (n_orders) n_orders[i] = env->n_orders[i];
        if (u_prev) u_prev[i] = env->u_prev[i];
        if (counts) {
            counts[3 * i + 0] = env->n_gather[i];
            counts[3 * i + 1] = env->n_craft[i];
            counts[3 * i + 2] = env->n_trade[i];
        }
        for (int r = 0; r < R; ++r) {
            if (inv) inv[i * R + r] = env->inv[i * R + r];
            if (inv_esc) inv_esc[i * R + r] = env->inv_esc[i * R + r];
        }
    }
}

int orc_env_get_book(const orc_env* env, int32_t* rows, int max_rows) {
    int n = env->n_book < max_rows ? env->n_book : max_rows;
    for (int k = 0; k < n; ++k) {
        const order_t* o = &env->book[k];
        int32_t* row = rows + 6 * k;
        row[0] = o->side; row[1] = o->r; row[2] = o->p;
        row[3] = o->agent; row[4] = o->step; row[5] = (int32_t)o->tb;
    }
    return env->n_book;
}

void orc_env_get_trades(const orc_env* env, int32_t* n_trades, int64_t* tick_volume) {
    for (int r = 0; r < env->prm.R; ++r) {
        if (n_trades) n_trades[r] = env->trades[r];
        if (tick_volume) tick_volume[r] = env->tick_volume[r];
    }
}
