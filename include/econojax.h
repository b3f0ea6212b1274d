/*
 * econojax.h - C ABI of the GB300 (sm_103a) EconoJax hot path.
 *
 * EconoJax (arxiv 2410.22165) is a vectorised economy: in each of E
 * environments, A population agents gather resources, craft them into coin
 * and trade them on a marketplace whose orders hold coin or units in escrow,
 * while a government agent sets bracketed tax rates each period and pays the
 * collected tax back in equal shares (Section 3).
 *
 * Conventions for every entry point:
 *  - Pointers marked (device) are CUDA device pointers; (host) are host
 *    pointers.  The caller allocates and owns all memory; no call allocates
 *    device memory.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = the legacy default stream).  They return after enqueueing.
 *  - Return value: EJ_OK, or an error code for invalid arguments (checked on
 *    the host before anything is enqueued; nothing runs) or a failed launch.
 *    ej_last_error() describes the most recent error of the calling thread.
 *  - Multi-dimensional arrays are dense, row-major, in the order written.
 *    E = environments, A = population agents per environment (the maximum
 *    when populations differ), n = steps.
 *
 * Environment rules (readings where the paper is silent are listed in the
 * repository's design notes):
 *  0. at a period start (t mod T_tax == 0) the government's rate levels take
 *     effect: rate_b = level_b / (tax_levels - 1)      (Sec. 3, "Setting tax rates")
 *  1. each agent's action is applied to its own state; an action the mask
 *     forbids does nothing                              (Sec. 3, "Population Agents",
 *                                                        "Action masking")
 *  2. per resource, the k-th best bid meets the k-th best ask while bid >= ask;
 *     priority: price, then age, then a random key; the trade is at the
 *     price of the newer order (the ask's when both are of the same step)
 *                                                       (Sec. 3 "Trading"; App. A)
 *  3. an order leaves after `expire` matching rounds; escrow goes back
 *  4. at a period end ((t+1) mod T_tax == 0) each agent pays the bracket tax
 *     on the period's earnings (at most its liquid coin); the total is paid
 *     back in equal shares                              (Sec. 3, "Setting tax rates")
 *  5. reward = change of isoelastic utility (Eq. 1-2) of coin incl. escrow;
 *     the government's = change of (omega(1-gini) + 1 - omega) * sum of coin (Eq. 3-5)
 *  6. after T_ep steps the environment restarts with new skills
 *  7. observation + action mask of the new state
 *
 * Action ids (nA = 2 + R + 2 R P):
 *   0 NO-OP | 1..R gather resource a-1 | R+1 craft |
 *   R+2 + r P + p   buy one unit of r at price level p |
 *   R+2 + R P + r P + p   sell one unit of r at price level p.
 * Mask: bit (a mod 32) of word a/32 is set when action a is allowed.
 *
 * Population observation (D = 8 + 7R + nb floats): coin, coin in escrow,
 * labor, inv[R], inv in escrow[R], gather skill[R], craft skill,
 * orders/max_orders, per resource {best bid, best ask (0 if none),
 * #bids/A_e, #asks/A_e}, rates[nb], period earnings, fraction of the tax
 * period left, t/T_ep.
 * Government observation (G = 9 + nb + 2): {mean, population std, median} of
 * {coin incl. escrow, period earnings, labor}, rates[nb], fraction of the tax
 * period left, t/T_ep.
 *
 * Random draws (Philox-4x32-10, key = 64-bit seed, low word first; Salmon et
 * al., SC'11).  Counter (c0, c1, c2, c3):
 *   population agent i of env e at global step g:  (i, e, g, 0) ->
 *       x0 uniform action floor(x0 nA / 2^32), x1 gather u, x2 tie-break key,
 *       x3 policy-sampling u
 *   government of env e at global step g:          (0, e, g, 1) ->
 *       x_b rate level floor(x_b tax_levels / 2^32) / policy u of bracket b
 *   skills of agent i, env e, episode k:           (i, e, k, 2 | c << 8) ->
 *       uniforms of chunks c = 0, 1, ... in order: SG[0..R-1], SC
 *   u = (x >> 8) * 2^-24.  g counts steps since env_reset across restarts.
 */
#ifndef ECONOJAX_H
#define ECONOJAX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EJ_MAX_A 1024        /* population agents per environment */
#define EJ_MAX_R 16          /* resource types */
#define EJ_MAX_P 32          /* price levels */
#define EJ_MAX_NB 4          /* tax brackets */
#define EJ_MAX_ORDERS 16     /* active orders per agent */
#define EJ_MAX_ACTIONS 256   /* 2 + R + 2 R P */
#define EJ_MAX_LEVELS 512    /* 2 R P order-book levels */

typedef enum {
    EJ_OK = 0,
    EJ_ERR_ARG = 1,          /* invalid argument; nothing was enqueued */
    EJ_ERR_CUDA = 2,         /* a CUDA call or launch failed */
    EJ_ERR_UNSUPPORTED = 3   /* valid but outside the compiled limits */
} ej_status;

/* Environment parameters.  Defaults (ej_params_default) are Table 2 of the
 * paper; craft_coin, thresholds and tax_levels are readings of values the
 * paper does not print. */
typedef struct {
    int32_t E;               /* environments */
    int32_t A;               /* population agents per environment (maximum) */
    int32_t R;               /* resource types (Table 2: 2) */
    int32_t P;               /* price levels (Table 2: 5) */
    int32_t nb;              /* tax brackets (3) */
    int32_t T_ep;            /* episode length (1000) */
    int32_t T_tax;           /* tax period (100) */
    int32_t expire;          /* matching rounds an order takes part in (30) */
    int32_t max_orders;      /* active orders per agent (15) */
    int32_t Rk;              /* craft: units needed per resource (2) */
    int32_t Rd;              /* craft: distinct resources needed (2) */
    int32_t allow_noop;      /* 1: NO-OP allowed (True) */
    int32_t gov_enabled;     /* 0: free market, no taxes */
    int32_t tax_levels;      /* rate levels per bracket (21: 0, 5, ..., 100 %) */
    float start_coin;        /* 15 */
    float eta;               /* isoelastic utility (0.27) */
    float omega;             /* equality weight (1) */
    float labor_gather;      /* 1 */
    float labor_craft;       /* 1 */
    float labor_trade;       /* 0.05 */
    float craft_coin;        /* coin per unit of craft skill (10) */
    float gather_rho;        /* gather draw range [0, gather_rho) (1.1) */
    float price_tick;        /* prices are whole multiples of this (2) */
    int32_t price_ticks[EJ_MAX_P];      /* level p costs price_tick*price_ticks[p]; ascending ({1..5}) */
    float thresholds[EJ_MAX_NB - 1];    /* bracket edges, ascending ({50, 100}) */
    /* Skill improvement (Section 5's multi-resource experiments; off in Table 2):
     * a gather raises that resource's gather skill, a craft the craft skill, by
     * s <- min(skill_max, s + s * skill_gain * (1 - s / skill_max)) in float32
     * (relative gain skill_gain, shrinking to 0 at skill_max).  READING of the
     * section's half-percent bonus that falls off towards the skill ceiling. */
    float skill_gain;        /* 0: skills fixed (Table 2); Section 5: 0.005 */
    float skill_max;         /* 5 */
    /* Skills at each episode start: 0 = U[0, 1) (Table 2); 1 = Section 5's
     * normally distributed skills of mean 1 and unit standard deviation, READ
     * as the Irwin-Hall sum of 12 uniforms - 5 (mean 1, variance exactly 1),
     * clamped to [0, skill_max]; uniform k of skill j is word k % 4 of the
     * Philox draw (i, e, episode, 2 | (3j + k / 4) << 8), summed in order in
     * float32. */
    int32_t skill_init;
} EjParams;

/* Sizes implied by a parameter set. */
typedef struct {
    int32_t n_actions;       /* nA */
    int32_t obs_dim;         /* D */
    int32_t gobs_dim;        /* G */
    int32_t mask_words;      /* W = ceil(nA / 32) */
    int32_t levels;          /* 2 R P */
    int32_t book_cap;        /* order slots per environment = A * max_orders */
    int32_t threads;         /* threads of the CTA that runs one environment */
    int32_t smem_bytes;      /* dynamic shared memory of that CTA */
    uint64_t state_bytes;    /* size of the state buffer */
} EjSizes;

/* Fields of the state buffer, for inspection (ej_state_field). */
typedef enum {
    EJ_F_COIN = 0,       /* float   [E][A_s]    liquid coin */
    EJ_F_ESC,            /* int32   [E][A_s]    coin in escrow, price ticks */
    EJ_F_INCOME,         /* float   [E][A_s]    earnings this tax period */
    EJ_F_UPREV,          /* float   [E][A_s]    utility after the previous step */
    EJ_F_NORD,           /* int32   [E][A_s]    active orders */
    EJ_F_COUNTS,         /* int32   [E][3][A_s] gathers, crafts, orders this episode */
    EJ_F_SC,             /* float   [E][A_s]    craft skill */
    EJ_F_INV,            /* int32   [E][R][A_s] liquid units */
    EJ_F_INVE,           /* int32   [E][R][A_s] units in escrow */
    EJ_F_SG,             /* float   [E][R][A_s] gather skill */
    EJ_F_T,              /* int32   [E]         step within the episode */
    EJ_F_GSTEP,          /* uint32  [E]         steps since env_reset */
    EJ_F_EPISODE,        /* uint32  [E]         episodes started since env_reset */
    EJ_F_POP,            /* int32   [E]         population A_e */
    EJ_F_RATES,          /* float   [E][4]      tax rates in effect */
    EJ_F_UGPREV,         /* float   [E]         social welfare after the previous step */
    EJ_F_LEVEL_COUNT,    /* int32   [E][L]      resting orders per book level */
    EJ_F_BOOK,           /* uint32  [E][cap]    orders: (placed step << 16) | agent,
                                                level after level, oldest first */
    EJ_F_KEY,            /* uint32  [2]         Philox key */
    EJ_F_COUNT_
} ej_field;

/* Writes the defaults of Table 2 (and the readings above) into *p, with E = 1
 * and A = 100. */
ej_status ej_params_default(EjParams* p);

/* Validates *p and fills *s.  EJ_ERR_ARG / EJ_ERR_UNSUPPORTED on bad values. */
ej_status ej_sizes(const EjParams* p, EjSizes* s);

/* Byte offset, element count and element size of a field of the state buffer.
 * A_s = A rounded up to a multiple of 4; book levels are ordered
 * l = (r * 2 + side) * P + p with side 0 = bids, 1 = asks. */
ej_status ej_state_field(const EjParams* p, int32_t field, uint64_t* offset,
                         uint64_t* count, int32_t* elem_bytes);

/* env_reset (Sec. 3 "Overall design": functional reset(key, params)).
 * state     (device) ej_sizes().state_bytes bytes, 256-byte aligned; written.
 * pop_sizes (device) int32[E] populations A_e in [1, A], or NULL for all A.
 * seed      Philox key for in-kernel draws (skills now and at restarts, and
 *           any draws env_step makes itself).
 * obs (device) float[E][A][D], gobs float[E][G], mask uint32[E][A][W]: the
 *           first observation; each may be NULL.  Rows of agents >= A_e are 0. */
ej_status env_reset(const EjParams* p, void* state, const int32_t* pop_sizes,
                    uint64_t seed, float* obs, float* gobs, uint32_t* mask,
                    void* stream);

/* env_step (Sec. 3 "Overall design": step(key, state, action, params)),
 * n_steps steps in one launch, state kept on chip between steps.
 * act      (device) int32[n][E][A] population actions (ids above), or NULL to
 *          draw uniform random actions in the kernel with the counter mapping
 *          above (then gather_u and tb must be NULL too).
 * gov_act  (device) int32[n][E][nb] rate levels (read at period starts only),
 *          or NULL to draw uniform levels in the kernel.
 * gather_u (device) float[n][E][A] gather draws u in [0,1); rho = gather_rho*u.
 * tb       (device) uint32[n][E][A] tie-break keys of orders placed that step.
 *          gather_u and tb are both given or both NULL (drawn in the kernel).
 * rew      (device) float[n][E][A] population rewards      (may be NULL)
 * grew     (device) float[n][E]    government rewards      (may be NULL)
 * done     (device) uint8[n][E]    1 when the step ended the episode (may be NULL)
 * obs, gobs, mask (device) as in env_reset, one per step [n][...] (may be NULL).
 * Out-of-range action ids act as forbidden actions; out-of-range rate levels
 * are clamped.  Integer state is exact; coin and utility are float32. */
ej_status env_step(const EjParams* p, void* state, int32_t n_steps,
                   const int32_t* act, const int32_t* gov_act,
                   const float* gather_u, const uint32_t* tb,
                   float* rew, float* grew, uint8_t* done,
                   float* obs, float* gobs, uint32_t* mask, void* stream);

/* env_step_host: env_step (Sec. 3 "Overall design") with every input and
 * output in HOST memory, for callers whose data lives on the host.
 * act, gov_act, gather_u, tb (host): as in env_step ([n][E][A] / [n][E][nb]),
 * each may be NULL under env_step's rules (in-kernel draws).
 * rew, grew, done, obs, gobs, mask (host): as in env_step, each may be NULL.
 * The steps run in chunks of `chunk` steps through two sets of staging
 * buffers in `workspace` (device, 256-byte aligned, at least
 * ej_step_host_workspace_bytes(p, chunk) bytes, caller-owned, no
 * initialisation needed): chunk k+1's inputs are copied in while chunk k
 * runs and chunk k-1's outputs are copied out, on three library-owned
 * streams that fork from `stream` and join back into it.  The call returns
 * after enqueueing; the host outputs are complete once `stream` has reached
 * this point (e.g. cudaStreamSynchronize).  Host arrays should be page-
 * locked (cudaHostAlloc, pinned tensors) for the copies to overlap the
 * kernel; pageable memory works but serialises them.  Results equal
 * env_step's bit for bit.  Calls on one device are enqueued one at a time
 * (internal lock).  Errors as env_step; EJ_ERR_ARG also for a NULL or too
 * small workspace, chunk < 1. */
ej_status ej_step_host_workspace_bytes(const EjParams* p, int32_t chunk, uint64_t* bytes);
ej_status env_step_host(const EjParams* p, void* state, int32_t n_steps, int32_t chunk,
                        const int32_t* act, const int32_t* gov_act, const float* gather_u, const uint32_t* tb,
                        float* rew, float* grew, uint8_t* done, float* obs, float* gobs, uint32_t* mask,
                        void* workspace, uint64_t workspace_bytes, void* stream);

/* ej_fill_draws: the draws env_step would make itself, written out (device),
 * for global steps g0 .. g0+n-1: act int32[n][E][A], gather_u float[n][E][A],
 * tb uint32[n][E][A], policy_u float[n][E][A], gov_act int32[n][E][nb];
 * each may be NULL.  Uses p->E, p->A and the counter mapping above. */
ej_status ej_fill_draws(const EjParams* p, uint64_t seed, uint32_t g0, int32_t n_steps,
                        int32_t* act, float* gather_u, uint32_t* tb, float* policy_u,
                        int32_t* gov_act, void* stream);

/* ------------------------------------------------------------------ policy
 * Actor and critic of Section 4: two hidden layers of `hidden` units with
 * ReLU, weights shared by all population agents (EJ_NET_POP: input D, one
 * head of nA logits, masked) and a separate pair for the government
 * (EJ_NET_GOV: input G, nb heads of tax_levels logits).  Parameter vector
 * (float32, row-major, y = x W + b, 16-byte aligned), in this order:
 *   W1 [in][H], b1 [H], W2 [H][H], b2 [H], W3 [H][O], b3 [O]      (actor)
 *   V1 [in][H], c1 [H], V2 [H][H], c2 [H], V3 [H], c3 [1]          (critic)
 * with O = nA (population) or nb * tax_levels (government); each tensor
 * starts at a multiple of 4 floats (the gaps are padding, ignored).
 * precision EJ_BF16: the five GEMMs on the tensor cores (tcgen05.mma, BF16
 * operands, FP32 accumulation in tensor memory), hidden in {64, 128};
 * EJ_FP32: float32 on the CUDA cores.
 * Sampling (Section 3 "Action masking": forbidden actions have probability 0)
 * is by inverse CDF on the masked softmax, computed in float32 with the
 * library's own exp (Cody-Waite reduction + degree-7 Taylor polynomial),
 * weights summed in action order; uniforms are x3 of the population counter
 * (i, e, g, 0) and x_b of the government counter (0, e, g, 1) at the state's
 * global step g, unless given. */
typedef enum { EJ_NET_POP = 0, EJ_NET_GOV = 1 } ej_net;
typedef enum { EJ_FP32 = 0, EJ_BF16 = 1 } ej_precision;

/* Floats of one network's parameter vector. hidden: multiple of 32 in [32, 256]. */
ej_status ej_net_floats(const EjParams* p, int32_t net, int32_t hidden, uint64_t* n_floats);

/* policy_forward: actor + critic over every row of the current state, and a
 * sampled action per row.
 * state   (device) the environment state (read: global step, Philox key).
 * weights (device) float[ej_net_floats].
 * obs     (device) float[E][A][D] (population) or float[E][G] (government).
 * mask    (device) uint32[E][A][W] (population; NULL: all allowed), ignored for the government.
 * u       (device) float[rows][heads] sampling uniforms, or NULL (Philox, above).
 * act     (device) int32[E][A] or int32[E][nb]; NULL: no sampling (values only).
 * logp, entropy (device) float[rows] (sum over heads); value float[rows];
 * logits  (device) float[rows][O] (may be NULL).  Rows with no allowed action
 * get action 0, logp 0, entropy 0.
 * BF16 takes hidden 64 or 128, at most 64 inputs and at most 128 logits with
 * (logits | 1) <= hidden (so <= 63 logits at hidden 64), and hidden 256 (the
 * networks of Section 5) with at most 64 inputs and 64 logits (a tile is
 * shared by the two CTAs of a thread-block cluster, each holding half of the
 * second layer's weights); other shapes return EJ_ERR_UNSUPPORTED (FP32 takes
 * them).  FP32 takes every shape: 64-row tiles (inputs, two hidden-width
 * buffers, logits twice) where they fit shared memory, 32-row tiles otherwise
 * (which fit up to hidden 256 with the largest market: 123 inputs, 242
 * logits). */
ej_status policy_forward(const EjParams* p, const void* state, int32_t net, int32_t hidden,
                         int32_t precision, const float* weights, const float* obs,
                         const uint32_t* mask, const float* u, int32_t* act, float* logp,
                         float* value, float* entropy, float* logits, void* stream);

/* policy_forward_segments: policy_forward over n_seg row sets in as few
 * launches as the kernels allow, e.g. the population and government
 * networks of several environment classes of a batch of uneven populations.
 * Set k: params[k], states[k] (device), nets[k] (EJ_NET_POP / EJ_NET_GOV),
 * weights[k] (device), obs[k], mask[k], act[k], logp[k], value[k] as in
 * policy_forward (the mask, act and logp arrays may be NULL, and so may their
 * entries; a government set takes no mask).  hidden and precision are common.
 * In BF16 with hidden 128, sets whose network has <= 96 logits and <= 32
 * inputs share launches: up to 4 networks (sets with the same weights
 * pointer, network and shape) and 32 sets per launch, CTAs split between
 * them by rows; other sets get a launch each.  Results equal separate
 * policy_forward calls.  Host arrays are read during the call only. */
ej_status policy_forward_segments(int32_t n_seg, const EjParams* const* params, const void* const* states,
                                  const int32_t* nets, const float* const* weights, int32_t hidden,
                                  int32_t precision, const float* const* obs, const uint32_t* const* mask,
                                  int32_t* const* act, float* const* logp, float* const* value, void* stream);

/* policy_segmented: *ok (host) = 1 when policy_forward_segments puts sets
 * of this network shape (params' observation / action sizes, net, hidden,
 * precision) into shared launches, else 0 (one launch per set). */
ej_status policy_segmented(const EjParams* p, int32_t net, int32_t hidden, int32_t precision, int32_t* ok);

/* Network layouts of the population (Section 5's three multi-agent methods):
 *   EJ_NETS_SHARED       one actor and one critic shared by all agents
 *                        (centralised training; Section 4's setting);
 *   EJ_NETS_INDEPENDENT  every agent its own actor and critic (iPPO);
 *   EJ_NETS_CTDE         every agent its own actor, one critic for all (the
 *                        section's naive CTDE / MAPPO: the critic sees the
 *                        same per-agent observation as the actor).
 * A per-agent population network is A consecutive parameter vectors of
 * ej_net_floats(EJ_NET_POP) floats each (the layout above): agent i's actor
 * is vector i's actor part; its critic is vector i's critic part
 * (independent) or vector 0's (CTDE, whose other critic parts are unused and
 * get zero gradients).  The government network stays one shared vector.
 * The forward and the rollout take FP32 or BF16 (BF16: hidden 64, 128 or 256; the
 * tensor-core kernel walks agent-major tiles, a contiguous range per CTA, and
 * packs an agent's weights when its tiles begin); the PPO gradient and update
 * of per-agent networks are FP32 (EJ_BF16 returns EJ_ERR_UNSUPPORTED). */
typedef enum { EJ_NETS_SHARED = 0, EJ_NETS_INDEPENDENT = 1, EJ_NETS_CTDE = 2 } ej_net_layout;

/* policy_forward of the population network under `layout` (EJ_NETS_SHARED:
 * policy_forward).  weights (device) A * ej_net_floats floats for a per-agent
 * layout; the other arguments as policy_forward's for EJ_NET_POP.  Rows of
 * agent i use agent i's actor and critic as the layout defines; sampled
 * actions follow the same counters. */
ej_status policy_forward_agents(const EjParams* p, const void* state, int32_t layout, int32_t hidden,
                                int32_t precision, const float* weights, const float* obs, const uint32_t* mask,
                                const float* u, int32_t* act, float* logp, float* value, float* entropy,
                                float* logits, void* stream);

/* Rollout buffer (device pointers, caller-owned).  Slot 0 of obs, gobs and
 * mask must hold the current observation (from env_reset or the previous
 * rollout's slot T). */
typedef struct {
    float* obs;          /* [T+1][E][A][D] */
    float* gobs;         /* [T+1][E][G] */
    uint32_t* mask;      /* [T+1][E][A][W] */
    int32_t* act;        /* [T][E][A] */
    int32_t* gact;       /* [T][E][nb] */
    float* logp;         /* [T][E][A] */
    float* glogp;        /* [T][E] */
    float* value;        /* [T+1][E][A]  (slot T: bootstrap value) */
    float* gvalue;       /* [T+1][E] */
    float* rew;          /* [T][E][A] */
    float* grew;         /* [T][E] */
    uint8_t* done;       /* [T][E] */
} EjRollout;

/* rollout: the data collection of PPO training (Section 4: the agents act
 * in E parallel environments for T steps with the current shared networks,
 * Table 2's rollout length; Section 3 "Overall design": the environment is
 * stepped as a pure function of state and actions).  T steps of {population
 * policy, government policy, env_step}, then the critics on slot T, on
 * `stream` (capture them in a CUDA graph to replay): 3T + 2 launches, or
 * 2T + 1 in BF16 where one launch serves both networks (per chain: from
 * E = 2048 on, rollout_split with 2 chains).  Gather draws and tie-break keys
 * come from the kernel's Philox streams.  Every member of buf is required
 * (EJ_ERR_ARG otherwise). */
ej_status rollout(const EjParams* p, void* state, int32_t T, int32_t hidden, int32_t precision,
                  const float* pop_weights, const float* gov_weights, const EjRollout* buf,
                  void* stream);

/* rollout_agents: rollout with the population's networks in `layout`
 * (EJ_NETS_SHARED: rollout itself); pop_weights as policy_forward_agents'.
 * One chain of 3T + 2 launches on `stream`. */
ej_status rollout_agents(const EjParams* p, void* state, int32_t T, int32_t hidden, int32_t precision,
                         int32_t layout, const float* pop_weights, const float* gov_weights, const EjRollout* buf,
                         void* stream);

/* rollout_split (Section 4, as rollout): rollout with the environments split into n_chains (1..4)
 * contiguous ranges whose T-step chains are independent (environments do
 * not interact), issued on as many streams: the caller's stream and library-
 * owned ones that fork from it and join back into it before the call
 * returns (so the result is ordered on `stream`, and a capture of `stream`
 * holds all chains).  One chain's env_step runs while another's policy
 * does.  Results equal rollout's bit for bit (draws are per environment). */
ej_status rollout_split(const EjParams* p, void* state, int32_t T, int32_t hidden, int32_t precision,
                        const float* pop_weights, const float* gov_weights, const EjRollout* b, int32_t n_chains,
                        void* stream);

/* --------------------------------------------------------------------- PPO
 * Clipped PPO (Section 4; Table 2) for the population and the government
 * networks at once (simultaneous training, Section 4): GAE, then `epochs`
 * passes over `minibatches` shuffled minibatches, each an Adam step of both
 * networks.  Loss per minibatch (advantages normalised over the minibatch):
 *   -mean(min(r A, clip(r, 1-clip, 1+clip) A))
 *   + vf_coef * mean(0.5 max((v - R)^2, (v_old + clip(v - v_old, +-vclip) - R)^2))
 *   - ent_coef * mean(entropy),       r = exp(logp - logp_old), R = A + v_old.
 * Minibatch m of an epoch holds the rollout rows pi(p), p in
 * [floor(m N / M), floor((m+1) N / M)), N = T * rows per step, where pi is
 * the Feistel permutation of [0, N) (4 rounds on b = max(2, ceil(log2 N))
 * bits: a high part of b / 2 bits and a low part of the rest, each round
 * XORing the part that is not its input with Philox word x0 of counter
 * (input part, round, shuffle_ctr, 4) masked to that part's width and
 * swapping the parts; cycle walking into [0, N)) keyed by `seed`.  ppo_update uses shuffle_ctr = update_index *
 * epochs + epoch for the population, with bit 31 set for the government. */
typedef struct {
    float gamma;         /* discount (0.99) */
    float lam;           /* GAE lambda (0.95) */
    float clip;          /* ratio clip (0.2) */
    float vf_coef;       /* value-loss coefficient (0.25) */
    float vclip;         /* value clip (10) */
    float ent_coef;      /* entropy coefficient (0.1; the caller anneals it) */
    float lr;            /* Adam learning rate (5e-4; the caller anneals it) */
    float beta1, beta2, eps;   /* Adam (0.9, 0.999, 1e-5) */
    int32_t epochs;      /* 4 */
    int32_t minibatches; /* 8; at most T x E, so that every minibatch of the
                          * government network holds a row (EJ_ERR_ARG otherwise) */
    uint64_t seed;       /* key of the minibatch shuffles */
} EjPpoParams;

ej_status ej_ppo_params_default(EjPpoParams* pp);

/* Bytes of the workspace the PPO calls need (caller-allocated, 256-byte
 * aligned, contents need no initialisation).  hidden: a multiple of 32 in
 * [32, 256] (Section 5's networks have 256 units).  The BF16 gradient takes
 * hidden 128 (at most 63 inputs, 64 logits, 4 heads, 2 mask words); the FP32
 * gradient takes every width, its 32-row tile (inputs, three hidden-width
 * buffers, logits) fitting shared memory at any shape the calls take (inputs
 * and logits at most 128).  Other shapes return EJ_ERR_UNSUPPORTED from the
 * gradient and update calls before anything runs. */
ej_status ej_ppo_workspace_bytes(const EjParams* p, const EjPpoParams* pp, int32_t T,
                                 int32_t hidden, uint64_t* bytes);

/* Byte offsets in the workspace of the advantages and returns (float
 * [T][rows]) of the population and the government: offsets[4] = {adv_pop,
 * ret_pop, adv_gov, ret_gov} (for inspection). */
ej_status ej_ppo_workspace_offsets(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                                   uint64_t* offsets);

/* GAE of both networks from a filled rollout buffer into the workspace:
 * A_t = d_t + gamma lam (1 - done_t) A_{t+1}, d_t = r_t + gamma (1 - done_t) V_{t+1} - V_t. */
ej_status ppo_advantages(const EjParams* p, const EjPpoParams* pp, int32_t T, const EjRollout* buf,
                         void* workspace, void* stream);

/* Gradient of one minibatch's loss for one network (net: EJ_NET_POP or
 * EJ_NET_GOV) into grad (device float[ej_net_floats], padding zeroed), after
 * ppo_advantages.  stats_out (device double[8], may be NULL): sums over the
 * minibatch of {advantage, advantage^2, policy loss, value loss, entropy,
 * clipped indicator, logp_old - logp}, then [7] the minibatch's loss itself,
 * (policy loss + vf_coef value loss - ent_coef entropy) / rows.
 * The rollout-buffer arrays read: obs, mask, act, logp, value (population) or
 * gobs, gact, glogp, gvalue (government); ppo_advantages reads rew, value,
 * grew, gvalue, done.  A NULL one of these returns EJ_ERR_ARG (nothing runs). */
ej_status ppo_minibatch_grad(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                             int32_t precision, int32_t net, const float* weights,
                             const EjRollout* buf, void* workspace, uint32_t shuffle_ctr,
                             int32_t minibatch, float* grad, double* stats_out, void* stream);

/* Data-parallel form of the minibatch gradient (the exchange step of a
 * multi-GPU update; Section 4's loss over the union of the ranks' minibatch
 * rows).  Each rank runs ppo_advantages on its own rollout, then per
 * minibatch and network:
 *   ppo_minibatch_moments: moments (device double[3]) = {rows of this rank's
 *     minibatch, sum of their GAE advantages, sum of squares};
 *   the caller sums the moments over the ranks (an all-reduce);
 *   ppo_minibatch_grad_global: this rank's part of the gradient of the union
 *     minibatch's loss: advantages normalised with the summed moments, means
 *     taken over moments[0] rows.  Summed over the ranks (a second
 *     all-reduce) it is the gradient of the union minibatch; with one rank and
 *     its own moments it equals ppo_minibatch_grad.
 * Arguments and errors otherwise as ppo_minibatch_grad; stats_out holds this
 * rank's sums, and [7] this rank's part of the union minibatch's loss (the
 * sums divided by moments[0]; the ranks' parts add up to the loss). */
ej_status ppo_minibatch_moments(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t net,
                                const EjRollout* buf, void* workspace, uint32_t shuffle_ctr,
                                int32_t minibatch, double* moments, void* stream);
ej_status ppo_minibatch_grad_global(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                                    int32_t precision, int32_t net, const float* weights,
                                    const EjRollout* buf, void* workspace, uint32_t shuffle_ctr,
                                    int32_t minibatch, const double* moments, float* grad,
                                    double* stats_out, void* stream);

/* One Adam step (Kingma and Ba, 2015) over n parameters; step counts from 1. */
ej_status adam_step(uint64_t n, float* params, const float* grad, float* m, float* v, int32_t step,
                    float lr, float beta1, float beta2, float eps, void* stream);

/* The whole update: ppo_advantages, then epochs x minibatches x {population,
 * government} gradient + Adam step.  Adam moments m, v (device, zero before
 * the first update) as long as the parameter vectors; adam_steps_done = Adam
 * steps taken before this call.  stats_out (device float[2][8], may be NULL):
 * per network mean policy loss, value loss, entropy, clip fraction,
 * logp_old - logp over all minibatch rows of the update. */
ej_status ppo_update(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                     int32_t precision, float* pop_weights, float* gov_weights, float* pop_m,
                     float* pop_v, float* gov_m, float* gov_v, int32_t adam_steps_done,
                     uint32_t update_index, const EjRollout* buf, void* workspace,
                     float* stats_out, void* stream);

/* PPO with the population's networks in a per-agent layout (Section 5:
 * independent training, iPPO; CTDE / MAPPO), FP32 (EJ_BF16 returns
 * EJ_ERR_UNSUPPORTED).  EJ_NETS_SHARED makes each call the shared one above
 * (ej_ppo_workspace_bytes, ppo_minibatch_grad for EJ_NET_POP, ppo_update).
 * Each agent trains its own actor (and, independent, its own critic) on its
 * own transitions: minibatch m of an epoch is, for every agent i, the rows
 * pi(q) * A + i for q in [floor(m N / M), floor((m+1) N / M)), N = T * E,
 * with pi the Feistel permutation of [0, N) described above (same keys and
 * counters; one shuffle of the (step, environment) pairs serves all agents).
 * An actor's loss is the mean over its agent's rows, with advantages
 * normalised over them; a shared critic's (CTDE) loss is the mean over all
 * agents' rows.  Gradients, Adam moments and weights of the population are
 * A vectors (A * ej_net_floats floats; a CTDE critic lives in vector 0 and
 * the other vectors' critic parts get zero gradients).  stats_out of
 * ppo_minibatch_grad_agents: sums over all rows (entry 7: their mean loss).
 * The workspace (ej_ppo_workspace_bytes_agents) also serves ppo_advantages. */
ej_status ej_ppo_workspace_bytes_agents(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                                        int32_t layout, uint64_t* bytes);
ej_status ppo_minibatch_grad_agents(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                                    int32_t precision, int32_t layout, const float* weights, const EjRollout* buf,
                                    void* workspace, uint32_t shuffle_ctr, int32_t minibatch, float* grad,
                                    double* stats_out, void* stream);
ej_status ppo_update_agents(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden, int32_t precision,
                            int32_t layout, float* pop_weights, float* gov_weights, float* pop_m, float* pop_v,
                            float* gov_m, float* gov_v, int32_t adam_steps_done, uint32_t update_index,
                            const EjRollout* buf, void* workspace, float* stats_out, void* stream);

/* ppo_minibatch_grad_static: ppo_minibatch_grad for callers that cannot
 * allocate device memory: hosts whose device memory belongs to another
 * runtime's pool allocator, which hands out no extra buffers; C programs that
 * embed the library without a device allocator of their own; service loops
 * that must not allocate once they are running.  It needs no
 * workspace: the advantages of `net`, the activations and the split-K partial
 * sums live in a static device array of 48 MiB that the library holds on every
 * GPU that loads it, until the process exits.  It computes the advantages of
 * `net` itself (no ppo_advantages call), otherwise arguments, layout and the
 * gradient are those of ppo_minibatch_grad (the partial sums are reduced in
 * 16 chunks instead of 96, so results agree to rounding).  The paper has no
 * counterpart: this is a convenience of this library.
 * precision must be EJ_FP32 (EJ_BF16 returns EJ_ERR_UNSUPPORTED: the tensor-
 * core gradient keeps per-CTA accumulators that do not fit the array).
 * Limits: the rollout's advantages and one minibatch of activations must fit
 * 48 MiB (about 8 thousand minibatch rows at hidden 128); larger sizes return
 * EJ_ERR_UNSUPPORTED with the bytes needed, before anything is enqueued.
 * The first call on a device, with that device current, looks the array's
 * address up (cudaGetSymbolAddress): make it before any stream capture.
 * Every call shares the array and leaves its contents behind; calls that
 * overlap on the GPU race on it and must be serialised by the caller.
 * It calls no cudaMalloc, cudaFree or other allocating routine. */
ej_status ppo_minibatch_grad_static(const EjParams* p, const EjPpoParams* pp, int32_t T, int32_t hidden,
                                    int32_t precision, int32_t net, const float* weights,
                                    const EjRollout* buf, uint32_t shuffle_ctr, int32_t minibatch,
                                    float* grad, double* stats_out, void* stream);

/* Synchronous read of the device fault word: *fault != 0 when a bounded
 * wait of a tensor-core kernel gave up (the kernel then freed its tensor
 * memory and returned without finishing).  clear != 0 resets it. */
ej_status ej_device_status(int32_t* fault, int32_t clear);

/* Description of the last error returned to the calling thread. */
const char* ej_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ECONOJAX_H */
