/*
 * CPU oracle of the EconoJax environment (arxiv 2410.22165, Section 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this code: it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can check the CUDA library against a plain,
 * slow, obviously correct statement of the rules.  It shares no code, header
 * or constant with the CUDA library; its parameter struct is its own.
 *
 * One orc_env is one environment.  All random draws (actions, gather draws,
 * tie-break keys, skills) are inputs: the caller supplies them.
 *
 * Precision: every reported quantity (coin, income, labor, utility, rewards,
 * observations, government statistics) is carried in double.  The values that
 * decide integer state (liquid coin against a price, the gather sum, the tax
 * that feeds liquid coin) are additionally carried in a float "decision
 * mirror" whose operations are spelled out one rounding at a time, because
 * the paper's own pipeline computes in float32 and integer state must not
 * depend on the precision of the machine that runs the rules.
 *
 * Parity pins: see the header of ej_oracle.c.
 */
#ifndef EJ_ORACLE_H
#define EJ_ORACLE_H
#include <stdint.h>

#define ORC_MAX_R 16
#define ORC_MAX_P 32
#define ORC_MAX_NB 8

typedef struct {
    int R;            /* resource types (Section 3, "Collecting resources") */
    int P;            /* price levels (Table 2: 5 prices) */
    int nb;           /* tax brackets, nb-1 thresholds (Section 3, "Setting tax rates") */
    int T_ep;         /* episode length (Table 2: 1000) */
    int T_tax;        /* tax period length (Table 2: 100) */
    int expire;       /* matching rounds an order takes part in (Table 2: 30) */
    int max_orders;   /* active orders per agent (Table 2: 15) */
    int Rk, Rd;       /* craft requirement (Section 3, "Crafting"; Table 2: 2, 2) */
    int allow_noop;   /* Table 2: True */
    int gov_enabled;  /* government agent present (Section 4 compares with a free market) */
    int tax_levels;   /* number of rate levels: 21 gives 0%, 5%, ..., 100% */
    double start_coin, eta, omega;
    double labor_gather, labor_craft, labor_trade;
    double craft_coin;      /* coin per unit of crafting skill (unprinted constant) */
    double gather_rho;      /* upper end of the gather draw (1.1) */
    double price_tick;      /* all prices are integer multiples of this */
    int price_ticks[ORC_MAX_P];          /* level p costs price_tick * price_ticks[p], ascending */
    double thresholds[ORC_MAX_NB - 1];   /* bracket edges, ascending */
    /* Section 5's multi-resource experiments: a gather raises that gather
     * skill, a craft the craft skill, by 0.5 % shrinking to 0 at the maximum
     * skill 5 (READING: s + s * (gain * (1 - s / max)), capped; 0 = off). */
    double skill_gain, skill_max;
} orc_params;

typedef struct orc_env orc_env;

/* Sizes implied by the parameters. */
int orc_num_actions(const orc_params* p);
int orc_obs_dim(const orc_params* p);
int orc_gobs_dim(const orc_params* p);
int orc_mask_words(const orc_params* p);

orc_env* orc_env_new(const orc_params* p, int A);
void orc_env_free(orc_env* env);

/* Start an episode: skills sg[A*R] (agent-major) and sc[A] are the draws. */
void orc_env_reset(orc_env* env, const float* sg, const float* sc);

/* One step.  act[A], gov_act[nb], gather_u[A], tb[A] are this step's inputs.
 * If the step ends the episode, the environment restarts with the skills in
 * next_sg / next_sc (may be NULL otherwise).  Outputs: rew[A], *grew, *done,
 * obs[A*obs_dim], gobs[gobs_dim], mask[A*mask_words]; any may be NULL. */
void orc_env_step(orc_env* env, const int32_t* act, const int32_t* gov_act,
                  const float* gather_u, const uint32_t* tb,
                  const float* next_sg, const float* next_sc,
                  double* rew, double* grew, int32_t* done,
                  double* obs, double* gobs, uint32_t* mask);

/* Observation, government observation and mask of the current state. */
void orc_env_observe(const orc_env* env, double* obs, double* gobs, uint32_t* mask);

/* Run n steps with inputs laid out [n][A] (act, gather_u, tb) and [n][nb]
 * (gov_act); skills for later episodes are [n_episodes][A*R] and [n_episodes][A]
 * (episode k+1 uses row k).  Outputs are [n][...] and may be NULL. */
void orc_env_run(orc_env* env, int n, const int32_t* act, const int32_t* gov_act,
                 const float* gather_u, const uint32_t* tb,
                 const float* later_sg, const float* later_sc,
                 double* rew, double* grew, int32_t* done,
                 double* obs, double* gobs, uint32_t* mask);

/* State read-out (for tests).  Arrays are agent-major. */
typedef struct {
    int t, episode, n_book;
    float rates32[ORC_MAX_NB];
    double rates64[ORC_MAX_NB];
    double ug_prev;
} orc_env_info;
void orc_env_get_info(const orc_env* env, orc_env_info* info);
/* coin32[A], coin64[A], income32[A], income64[A], esc_ticks[A], inv[A*R],
 * inv_esc[A*R], n_orders[A], counts[A*3] (gather, craft, trade), u_prev[A];
 * any may be NULL. */
void orc_env_get_agents(const orc_env* env, float* coin32, double* coin64,
                        float* income32, double* income64, int32_t* esc_ticks,
                        int32_t* inv, int32_t* inv_esc, int32_t* n_orders,
                        int32_t* counts, double* u_prev);
/* Active orders, one row of 6 ints each: side (0 bid, 1 ask), resource, price
 * level, agent, placed step, tie-break key (as int32 bits). Returns count. */
int orc_env_get_book(const orc_env* env, int32_t* rows, int max_rows);
/* Market totals of the last step: trades per resource, summed trade ticks. */
void orc_env_get_trades(const orc_env* env, int32_t* n_trades, int64_t* tick_volume);

/* Closed-form helpers exposed for pinning. */
double orc_gini(const double* x, int n);
double orc_isoelastic(double coin, double labor, double eta);
double orc_bracket_tax(double income, const double* rates, const double* thresholds, int nb);

#endif
