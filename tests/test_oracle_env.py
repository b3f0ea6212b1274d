"""Pins of the CPU oracle against what the paper and the mathematics fix.

Runs without a GPU.  Each test names the passage it pins.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import env as oenv
from oracle.env import OracleEnv, default_params
from tests.oracle_scenarios import NOOP, Scenario, buy, craft, gather, sell

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generator

def test_philox_known_answers():
    """Philox-4x32-10 against the vectors published with its definition (SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = synth.philox4x32_10(*v[:6])
        assert [int(x) for x in out] == v[6:]


def test_uniform_maps():
    x = np.array([0, 255, 256, 0xFFFFFFFF], dtype=np.uint32)
    u = synth.u01(x)
    assert u.dtype == np.float32
    assert list(u) == [0.0, 0.0, 2.0 ** -24, 1.0 - 2.0 ** -24]
    assert list(synth.below(x, 24)) == [0, 0, 0, 23]


# ------------------------------------------------------------ action layout

@pytest.mark.parametrize("R,P,n", [(4, 3, 30), (12, 3, 86), (2, 5, 24)])
def test_action_counts(R, P, n):
    """Section 5: 30 actions at 4 resources and 86 at 12, with three prices and NO-OP."""
    assert oenv.num_actions(default_params(R=R, P=P, price_ticks=list(range(1, P + 1)))) == n


def test_sizes_default():
    p = default_params()
    assert oenv.obs_dim(p) == 25 and oenv.gobs_dim(p) == 14 and oenv.mask_words(p) == 1


# ------------------------------------------------------------- closed forms

def test_gini_closed_forms():
    """Gini index: 0 for equality, (n-1)/n when one holds everything,
    (n-1)/(3n) for the values 1..n (mean absolute difference (n^2-1)/(3n))."""
    for n in (1, 2, 7, 100):
        assert oenv.gini(np.full(n, 3.5)) == 0.0
        x = np.zeros(n); x[-1] = 42.0
        assert oenv.gini(x) == pytest.approx((n - 1) / n, abs=1e-12)
        assert oenv.gini(np.arange(1, n + 1, dtype=float)) == pytest.approx((n - 1) / (3 * n), abs=1e-12)
    assert oenv.gini(np.zeros(5)) == 0.0


def test_isoelastic_properties():
    """Eq. 1: zero at one coin and no labor; labor enters one for one; marginal
    utility C^-eta; tends to ln C as eta -> 1 (the textbook limit)."""
    eta = 0.27
    assert oenv.isoelastic(1.0, 0.0, eta) == pytest.approx(0.0, abs=1e-15)
    assert oenv.isoelastic(20.0, 3.0, eta) == pytest.approx(oenv.isoelastic(20.0, 0.0, eta) - 3.0)
    for c in (0.5, 15.0, 400.0):
        h = 1e-5 * c
        d = (oenv.isoelastic(c + h, 0, eta) - oenv.isoelastic(c - h, 0, eta)) / (2 * h)
        assert d == pytest.approx(c ** -eta, rel=1e-7)
        assert oenv.isoelastic(c, 0.0, 1.0 - 1e-9) == pytest.approx(math.log(c), abs=1e-6)


def test_tax_worked_example_closed_form():
    g = json.load(open(os.path.join(GOLDEN, "tax_worked_example.json")))
    rates = [l / (g["tax_levels"] - 1) for l in g["rate_levels"]]
    assert oenv.bracket_tax(g["income"], rates, g["thresholds"]) == pytest.approx(g["tax"], abs=1e-12)
    # below the first edge only the first rate applies; zero earnings pay nothing
    assert oenv.bracket_tax(40.0, rates, g["thresholds"]) == pytest.approx(4.0)
    assert oenv.bracket_tax(0.0, rates, g["thresholds"]) == 0.0


def test_tax_worked_example_through_the_environment():
    """Section 3: the agent that earned 130 pays 35 at the period end and gets
    1/n of the pool back; the other agent only receives its share."""
    g = json.load(open(os.path.join(GOLDEN, "tax_worked_example.json")))
    s = Scenario(2, sg=[[2.0, 2.0], [1.0, 1.0]], sc=[13.0, 0.5], T_tax=10,
                 thresholds=g["thresholds"], tax_levels=g["tax_levels"])
    s.step([gather(0), NOOP], gov=g["rate_levels"])
    s.step([gather(1), NOOP])
    s.step([craft(), NOOP])
    a = s.agents()
    assert a["income64"][0] == 130.0 and a["income32"][0] == np.float32(130.0)
    for _ in range(7):
        s.step([NOOP, NOOP])
    a = s.agents()
    share = g["tax"] / 2
    assert a["coin64"][0] == pytest.approx(15 + 130 - g["tax"] + share, abs=1e-12)
    assert a["coin64"][1] == pytest.approx(15 + share, abs=1e-12)
    assert a["coin32"][0] == np.float32(127.5) and a["coin32"][1] == np.float32(32.5)
    assert a["income64"][0] == 0.0


def test_tax_capped_at_liquid_coin():
    """READING (paper silent): tax cannot exceed the coin outside escrow."""
    s = Scenario(2, sg=[[2.0, 2.0], [1.0, 1.0]], sc=[13.0, 0.5], T_tax=10)
    s.step([gather(0), NOOP], gov=[20, 20, 20])
    s.step([gather(1), NOOP])
    s.step([craft(), NOOP])
    for _ in range(7):
        s.step([buy(0, 4), NOOP])        # 7 resting bids of 10: 70 coin in escrow
    a = s.agents()
    assert a["esc_ticks"][0] == 35
    assert a["coin64"][0] == pytest.approx(37.5) and a["coin64"][1] == pytest.approx(52.5)


# ---------------------------------------------------------------- gathering

def test_gather_boundaries_and_mean():
    """Section 3: floor(SG + rho), rho uniform in [0, 1.1): low skill can still
    gather, high skill can gather two; the mean is (0.1 + SG)/1.1 +
    max(0, SG - 0.9)/1.1."""
    n = 4000
    u = synth.u01(synth.philox4x32_10(np.arange(n), 7, 7, 7, 1, 2)[0])
    for sgv in (0.0, 0.3, 0.95):
        s = Scenario(n, sg=np.full((n, 2), sgv), T_ep=1000)
        s.step(np.full(n, gather(0)), u=u)
        amt = s.agents()["inv"][:, 0]
        assert set(np.unique(amt)) <= {0, 1, 2}
        mean = (0.1 + sgv) / 1.1 + max(0.0, sgv - 0.9) / 1.1
        assert abs(amt.mean() - mean) < 4 * math.sqrt(0.25 / n) + 1e-3
        assert amt.min() == 0 and (amt.max() == 2) == (sgv > 0.9)


# ------------------------------------------------------------------- market

def test_same_step_trade_at_ask_price():
    """App. A: price of the newer order; READING: the ask's price when
    both orders come in the same step."""
    s = Scenario(2)
    s.step([NOOP, gather(0)])
    s.step([buy(0, 4), sell(0, 0)])
    a = s.agents()
    assert a["coin64"].tolist() == [13.0, 17.0]
    assert a["inv"][:, 0].tolist() == [1, 0] and a["inv_esc"].sum() == 0
    assert a["esc_ticks"].tolist() == [0, 0] and a["n_orders"].tolist() == [0, 0]
    assert a["income64"].tolist() == [0.0, 2.0]
    n, v = s.env.trades()
    assert n[0] == 1 and v[0] == 1


def test_later_bid_sets_price():
    """App. A: a resting ask met by a later bid trades at the bid's price."""
    s = Scenario(2)
    s.step([NOOP, gather(0)])
    s.step([NOOP, sell(0, 2)])
    assert s.agents()["inv_esc"][1, 0] == 1
    s.step([buy(0, 4), NOOP])
    a = s.agents()
    assert a["coin64"].tolist() == [5.0, 25.0] and a["inv"][0, 0] == 1


def test_best_ask_first():
    """Section 3: low asks are evaluated first."""
    s = Scenario(3)
    s.step([NOOP, gather(0), gather(0)])
    s.step([NOOP, sell(0, 1), NOOP])
    s.step([NOOP, NOOP, sell(0, 0)])
    s.step([buy(0, 4), NOOP, NOOP])
    a = s.agents()
    assert a["coin64"].tolist() == [5.0, 15.0, 25.0]
    assert a["inv_esc"][:, 0].tolist() == [0, 1, 0]


def test_older_order_first():
    """Section 3: ties in price go to the older order (agent 2 placed first)."""
    s = Scenario(3)
    s.step([NOOP, gather(0), gather(0)])
    s.step([NOOP, NOOP, sell(0, 1)])
    s.step([NOOP, sell(0, 1), NOOP])
    s.step([buy(0, 1), NOOP, NOOP])
    a = s.agents()
    assert a["coin64"].tolist() == [11.0, 15.0, 19.0]
    assert a["inv_esc"][:, 0].tolist() == [0, 1, 0]


@pytest.mark.parametrize("keys,winner", [([0, 500, 100], 2), ([0, 100, 500], 1)])
def test_random_key_breaks_equal_age(keys, winner):
    """Section 3: a tie in price and age is broken by the random key (the smaller key first)."""
    s = Scenario(3)
    s.step([NOOP, gather(0), gather(0)])
    s.step([NOOP, sell(0, 1), sell(0, 1)], tb=keys)
    s.step([buy(0, 1), NOOP, NOOP])
    a = s.agents()
    assert a["inv_esc"][winner, 0] == 0 and a["inv_esc"][3 - winner, 0] == 1
    assert a["coin64"][winner] == 19.0


def test_no_trade_below_ask():
    s = Scenario(2)
    s.step([NOOP, gather(0)])
    s.step([buy(0, 0), sell(0, 1)])
    a = s.agents()
    assert a["esc_ticks"][0] == 1 and a["inv_esc"][1, 0] == 1
    assert len(s.env.book()) == 2 and s.env.trades()[0][0] == 0


def test_kth_best_pairing():
    """Bids [10, 4] against asks [2, 6]: the best pair trades, the second does not."""
    s = Scenario(4)
    s.step([NOOP, NOOP, gather(0), gather(0)])
    s.step([buy(0, 4), buy(0, 1), sell(0, 0), sell(0, 2)])
    a = s.agents()
    assert a["coin64"].tolist() == [13.0, 11.0, 17.0, 15.0]
    assert s.env.trades()[0][0] == 1 and len(s.env.book()) == 2


def test_two_pairs_each_at_the_later_price():
    s = Scenario(4)
    s.step([NOOP, NOOP, gather(0), gather(0)])
    s.step([NOOP, NOOP, sell(0, 0), sell(0, 1)])
    s.step([buy(0, 4), buy(0, 3), NOOP, NOOP])
    a = s.agents()
    assert a["coin64"].tolist() == [5.0, 7.0, 25.0, 23.0]
    assert a["inv"][:, 0].tolist() == [1, 1, 0, 0]


def test_resources_trade_separately():
    s = Scenario(2)
    s.step([NOOP, gather(1)])
    s.step([buy(0, 4), sell(1, 0)])
    assert s.env.trades()[0].tolist() == [0, 0] and len(s.env.book()) == 2


@pytest.mark.parametrize("side", ["ask", "bid"])
def test_expiry_after_expire_rounds(side):
    """Table 2 expire time: an order takes part in `expire` matching rounds
    (READING), then its escrow goes back."""
    s = Scenario(1, expire=3)
    s.step([gather(0)])
    s.step([sell(0, 4) if side == "ask" else buy(0, 0)])   # placed at step 1
    s.step([NOOP])                                          # round 2
    assert len(s.env.book()) == 1
    s.step([NOOP])                                          # round 3, then it expires
    a = s.agents()
    assert len(s.env.book()) == 0 and a["n_orders"][0] == 0
    assert a["inv"][0, 0] == 1 and a["inv_esc"][0, 0] == 0
    assert a["coin64"][0] == 15.0 and a["esc_ticks"][0] == 0


# ------------------------------------------------------------------ masking

def test_initial_mask_and_masked_action_is_noop():
    """Section 3 'Action masking': sell needs a unit, craft needs R_k of R_d
    resources, buy needs the price in coin; a masked action does nothing."""
    s = Scenario(1)
    obs, gobs, mask = s.env.observe()
    assert mask[0, 0] == 0x3FF7                 # NO-OP, gathers, ten buys
    s.step([sell(0, 0)])
    s.step([craft()])
    a = s.agents()
    assert a["counts"].tolist() == [[0, 0, 0]] and a["n_orders"][0] == 0
    s2 = Scenario(1, allow_noop=0)
    assert s2.env.observe()[2][0, 0] == 0x3FF6


def test_order_limit_and_price_mask():
    s = Scenario(1, max_orders=2)
    s.step([buy(0, 0)])
    s.step([buy(1, 0)])
    m = s.env.observe()[2][0, 0]
    assert m == 0x7                              # only NO-OP and gathers left
    s.step([buy(0, 1)])                          # masked: no third order
    assert s.agents()["n_orders"][0] == 2
    s3 = Scenario(1)
    s3.step([buy(0, 4)])                         # 15 -> 5 coin: prices 6..10 masked
    m = s3.env.observe()[2][0, 0]
    assert [(m >> (4 + k)) & 1 for k in range(5)] == [1, 1, 0, 0, 0]


def test_craft_uses_richest_resources():
    """Section 3 'Crafting': R_d resources prioritised by the amount held."""
    s = Scenario(1, sg=[[2.0, 2.0, 2.0]], sc=[0.25], R=3, Rk=2, Rd=2)
    for r in (0, 1, 1, 2, 2, 2):
        s.step([gather(r)])
    s.step([craft(R=3)])
    a = s.agents()
    assert a["inv"][0].tolist() == [2, 2, 4]
    assert a["coin64"][0] == 15.0 + 2.5


# ------------------------------------------------------- episode structure

def test_episode_end_and_reset():
    T = 7
    s = Scenario(2, T_ep=T, T_tax=5)
    for t in range(T):
        out = s.step([gather(0), buy(0, 0)])
        assert out["done"] == int(t == T - 1)
    a = s.agents()
    assert s.env.info()["t"] == 0 and s.env.info()["episode"] == 1
    assert a["coin64"].tolist() == [15.0, 15.0] and a["inv"].sum() == 0 and len(s.env.book()) == 0
    assert out["obs"][0, 2] == 0.0                       # labor restarts


# ---------------------------------------------- invariants on random play

def _random_run(seed, A, T, **params):
    p = default_params(**params)
    env = OracleEnv(p, A)
    inp = synth.episode_inputs(seed, [0], A, p["R"], p["nb"], env.nA, p["tax_levels"], T, p["T_ep"])
    env.reset(inp["sg0"][0], inp["sc0"][0])
    return p, env, inp


@pytest.mark.parametrize("seed,A,T_tax", [(0, 10, 10), (1, 37, 13), (2, 64, 100)])
def test_conservation_and_book_invariants(seed, A, T_tax):
    """Escrow semantics of Section 3: coin only enters through crafting (taxes
    are paid back in full), units only through gathering and leave through
    crafting; escrow equals the open orders; the book is never crossed after
    matching; the number of trades is max_q min(#bids >= q, #asks <= q)."""
    T = 160
    p, env, inp = _random_run(seed, A, T, T_ep=1000, T_tax=T_tax)
    R, P, tick = p["R"], p["P"], p["price_tick"]
    ticks = np.array(p["price_ticks"])
    sc = inp["sc0"][0].astype(np.float64)
    prev = env.agents()
    prev_book = env.book()
    n_trades_seen = 0
    for t in range(T):
        act = inp["act"][t, 0]
        out = env.step(act, inp["gov_act"][t, 0], inp["gather_u"][t, 0], inp["tb"][t, 0])
        a = env.agents()
        book = env.book()
        d_counts = a["counts"] - prev["counts"]
        crafted = d_counts[:, 1] == 1
        # coin: total (liquid + escrow) grows by craft gains only
        tot_prev = prev["coin64"] + tick * prev["esc_ticks"]
        tot = a["coin64"] + tick * a["esc_ticks"]
        assert tot.sum() - tot_prev.sum() == pytest.approx(p["craft_coin"] * sc[crafted].sum(), abs=1e-9)
        # units per resource: trades and escrow move units, they never make or
        # destroy them; gathering adds floor(SG + 1.1 u), crafting takes Rk
        units_prev = (prev["inv"] + prev["inv_esc"]).sum(0)
        units = (a["inv"] + a["inv_esc"]).sum(0)
        gathered = np.zeros(R, np.int64)
        for i in np.nonzero(d_counts[:, 0])[0]:
            r = act[i] - 1
            rho = np.float32(p["gather_rho"]) * inp["gather_u"][t, 0, i]
            gathered[r] += int(np.floor(np.float32(inp["sg0"][0][i, r]) + np.float32(rho)))
        assert (units - units_prev).tolist() == (gathered - p["Rk"] * crafted.sum()).tolist()
        # escrow and order counts match the open orders
        for i in range(A):
            mine = book[book[:, 3] == i]
            assert a["n_orders"][i] == len(mine)
            assert a["esc_ticks"][i] == ticks[mine[mine[:, 0] == 0, 2]].sum()
            for r in range(R):
                assert a["inv_esc"][i, r] == np.sum((mine[:, 0] == 1) & (mine[:, 1] == r))
        assert (a["inv"] >= 0).all() and (a["coin32"] >= 0).all() and (a["n_orders"] <= p["max_orders"]).all()
        # uncrossed book, and the count of trades
        new = [(int(j >= R * P), (j % (R * P)) // P, j % P) for i, j in
               ((i, act[i] - (R + 2)) for i in np.nonzero(d_counts[:, 2])[0])]
        n_tr, _ = env.trades()
        for r in range(R):
            bids = book[(book[:, 0] == 0) & (book[:, 1] == r), 2]
            asks = book[(book[:, 0] == 1) & (book[:, 1] == r), 2]
            if len(bids) and len(asks):
                assert bids.max() < asks.min()
            pre_b = [o[2] for o in prev_book if o[0] == 0 and o[1] == r] + [x[2] for x in new if x[0] == 0 and x[1] == r]
            pre_a = [o[2] for o in prev_book if o[0] == 1 and o[1] == r] + [x[2] for x in new if x[0] == 1 and x[1] == r]
            pre_b, pre_a = np.array(pre_b, int), np.array(pre_a, int)
            k = max(min(int((pre_b >= q).sum()), int((pre_a <= q).sum())) for q in range(P))
            assert n_tr[r] == k
            n_trades_seen += k
        prev, prev_book = a, book
    assert n_trades_seen > 0


@pytest.mark.parametrize("e", [0, 511])
def test_float_coin_within_the_coin_contract(e):
    """Float32 coin against the float64 track, per value and every step of a
    full episode of the benchmark workload (A = 100, 1000 steps, seed 1000).
    The GPU's coin equals the float mirror bit for bit, so this is the coin
    contract on the CPU.  READING of "1e-5 relative": relative to the larger of
    the value and the largest coin the agent has held since its episode began
    (a float sum keeps the absolute rounding error of the largest value it
    passed through); period earnings only grow within a period, so for them
    this is the value itself.  Liquid coin can fall to ~1 after ~100, and the
    plain per-value error (floor 1 coin) then exceeds 1e-5: printed, not
    asserted."""
    from tests.parity import coin_scale
    p = default_params()
    A, T = 100, 1000
    env = OracleEnv(p, A)
    inp = synth.episode_inputs(1000, [e], A, p["R"], p["nb"], env.nA, p["tax_levels"], T, p["T_ep"])
    env.reset(inp["sg0"][0], inp["sc0"][0])
    c32, c64, i32, i64 = (np.zeros((T - 1, A)) for _ in range(4))
    for t in range(T - 1):
        env.step(inp["act"][t, 0], inp["gov_act"][t, 0], inp["gather_u"][t, 0], inp["tb"][t, 0])
        a = env.agents()
        c32[t], c64[t], i32[t], i64[t] = a["coin32"], a["coin64"], a["income32"], a["income64"]
    scale = coin_scale(c64, np.zeros(T - 1, bool), p["start_coin"])
    err = np.abs(c32 - c64) / np.maximum(scale, 1.0)
    err_inc = np.abs(i32 - i64) / np.maximum(np.abs(i64), 1.0)
    plain = np.abs(c32 - c64) / np.maximum(np.abs(c64), 1.0)
    print(f"coin: {err.max():.2e} (contract scale), {plain.max():.2e} (plain per value); earnings {err_inc.max():.2e}")
    assert err.max() < 1e-5 and err_inc.max() < 1e-5


# ---- Section 5: skill improvement and the skill distribution around 1 ----

def _one_agent(s_gather, s_craft, acts, **kw):
    """One agent (R = 2, no taxes) taking the given actions with gather draws
    u = 0 (rho = 0); returns the observations [n, D] and the oracle."""
    p = default_params(T_ep=5000, T_tax=5000, gov_enabled=0, **kw)
    o = OracleEnv(p, 1)
    o.reset(np.array(s_gather, np.float32).reshape(1, 2), np.array([s_craft], np.float32))
    n = len(acts)
    out = o.run(np.array(acts, np.int32).reshape(n, 1), np.zeros((n, p["nb"]), np.int32),
                np.zeros((n, 1), np.float32), np.arange(n, dtype=np.uint32).reshape(n, 1))
    return out["obs"][:, 0, :], p


def test_skill_growth_is_logistic_and_uses_the_skill_before_the_step():
    """1200 gathers of resource 0 from skill 0.2 at gain 0.005, max 5: the
    skill follows K / (1 + (K/s0 - 1) (1 + g)^-n) (the logistic curve whose
    rate matches the 0.5 % gain at small skill) within 0.5 %; it never exceeds
    5; the other skills do not move; each gather brings floor(skill before the
    step) units (rho = 0)."""
    n, g, K, s0 = 1200, 0.005, 5.0, 0.2
    obs, p = _one_agent([s0, 0.7], 0.4, [1] * n, skill_gain=g, skill_max=K)
    R = 2
    sg0, sg1, sc = obs[:, 3 + 2 * R], obs[:, 3 + 2 * R + 1], obs[:, 3 + 3 * R]
    k = np.arange(1, n + 1)
    logistic = K / (1 + (K / s0 - 1) * (1 + g) ** (-k))
    assert np.max(np.abs(sg0 / logistic - 1)) < 5e-3
    assert (np.diff(sg0) >= 0).all() and sg0.max() <= K and sg0[-1] > 4.5
    assert (sg1 == np.float32(0.7)).all() and (sc == np.float32(0.4)).all()
    inv0 = obs[:, 3]
    before = np.concatenate([[np.float32(s0)], sg0[:-1]])
    assert np.array_equal(np.diff(np.concatenate([[0.0], inv0])), np.floor(before))


def test_skill_growth_fixed_points_and_cap():
    """Skill 0 stays 0; skill at the maximum stays there; a fast gain (0.6,
    maximum 2) reaches the maximum and never passes it."""
    R = 2
    obs, _ = _one_agent([0.0, 1.0], 0.0, [1] * 50, skill_gain=0.005)
    assert (obs[:, 3 + 2 * R] == 0).all()
    obs, _ = _one_agent([5.0, 1.0], 1.0, [1] * 50, skill_gain=0.005, skill_max=5.0)
    assert (obs[:, 3 + 2 * R] == np.float32(5.0)).all()
    obs, _ = _one_agent([1.9, 1.0], 1.0, [1] * 200, skill_gain=0.6, skill_max=2.0)
    assert obs[:, 3 + 2 * R].max() <= 2.0 and obs[-1, 3 + 2 * R] == np.float32(2.0)


def test_craft_skill_grows_by_the_same_rule():
    """With R_k = 0 crafting is always allowed: n crafts move the craft skill
    along exactly the trajectory n gathers give a gather skill from the same
    start (the same rule for both skills)."""
    R, n = 2, 300
    g_obs, _ = _one_agent([0.3, 1.0], 2.0, [1] * n, skill_gain=0.005, Rk=0)
    c_obs, _ = _one_agent([1.0, 1.0], 0.3, [R + 1] * n, skill_gain=0.005, Rk=0)
    assert np.array_equal(g_obs[:, 3 + 2 * R], c_obs[:, 3 + 3 * R])
    assert c_obs[-1, 3 + 3 * R] > 0.3


def test_skill_init_around_one():
    """Skill init 1: 12 uniforms summed minus 5, clamped to [0, 5]: median 1,
    interquartile range 1.349 (that of a unit normal), Phi(-1) of the skills
    clamped to 0, none above 5; init 0 stays U[0, 1)."""
    sg, sc = synth.skill_draws(7, np.arange(200), 100, 3, 4, init=1)
    v = np.concatenate([sg.ravel(), sc.ravel()]).astype(np.float64)
    assert v.min() >= 0.0 and v.max() <= 5.0
    assert abs(np.median(v) - 1.0) < 0.02
    q1, q3 = np.quantile(v, [0.25, 0.75])
    assert abs((q3 - q1) - 1.349) < 0.03
    assert abs((v == 0).mean() - 0.1587) < 0.006
    sg, sc = synth.skill_draws(7, np.arange(200), 100, 3, 4, init=0)
    u = np.concatenate([sg.ravel(), sc.ravel()])
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
