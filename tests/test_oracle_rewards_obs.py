"""Hand-worked pins of the oracle's reward composition, social welfare and
observation statistics (Section 3, Eq. 1-5; Fig. 1 caption; App. A).

Runs without a GPU.  Every expected value below is worked out by hand from
the scenario written next to it; none is produced by the oracle or the CUDA
library.  With eta = 0.5 the isoelastic utility of Eq. 1 is 2 (sqrt(C) - 1) - L,
so the expected rewards are sums of square roots of whole numbers.
"""
import math

import numpy as np
import pytest

from tests.oracle_scenarios import NOOP, Scenario, buy, craft, gather, sell

# population observation columns at R = 2, nb = 3 (25 floats)
COIN, ESC, LABOR, INV0, INV1, INVE0, INVE1, SG0, SG1, SC, NORD = range(11)
MKT = 11                          # per resource: best bid, best ask, #bids / A, #asks / A
RATES, INCOME, PLEFT, TFRAC = 19, 22, 23, 24
# government observation: {mean, std, median} of coin incl. escrow, earnings, labor
G_COIN, G_INC, G_LAB, G_RATES, G_PLEFT, G_TFRAC = 0, 3, 6, 9, 12, 13


def u_half(C, L):
    """Eq. 1 at eta = 0.5."""
    return 2.0 * (math.sqrt(C) - 1.0) - L


def _market_scenario(**kw):
    """Two agents, free market, one unit per resource per craft.  Start coin 16,
    prices 2, 4, 6, 8, 10 (tick 2), skills SG = 1 (u = 0 gathers exactly one
    unit), SC = 0.5 (agent 0) and 0.25 (agent 1), orders live 2 rounds."""
    params = dict(eta=0.5, start_coin=16.0, Rk=1, Rd=2, gov_enabled=0, expire=2)
    params.update(kw)
    s = Scenario(2, sg=[[1.0, 1.0], [1.0, 1.0]], sc=[0.5, 0.25], **params)
    out = []
    out.append(s.step([gather(0), NOOP]))                    # t0
    out.append(s.step([gather(1), gather(0)]))               # t1
    out.append(s.step([craft(), sell(0, 2)]))                # t2: agent 1 asks 6 for its unit
    out.append(s.step([buy(0, 4), NOOP]))                    # t3: agent 0 bids 10: trade at 10
    out.append(s.step([buy(1, 0), NOOP]))                    # t4: a bid of 2 rests (no asks)
    out.append(s.step([NOOP, NOOP]))                         # t5: that bid expires
    return s, out


def test_population_rewards_hand_worked():
    """Eq. 2 on Eq. 1: r = u(coin + escrow, labor) - u(previous step).
    Labor: 1 per gather or craft, 0.05 charged when an order is placed; coin
    in escrow still counts (a resting bid leaves utility unchanged apart from
    its labor); an expiring order moves coin back without changing utility."""
    _, out = _market_scenario()
    r = np.array([o["rew"] for o in out])
    s21, s11, s26 = math.sqrt(21), math.sqrt(11), math.sqrt(26)
    expect = np.array([
        [-1.0, 0.0],                                         # gather: one unit of labor
        [-1.0, -1.0],
        [2 * s21 - 9.0, -0.05],                              # craft +5 coin, +1 labor; ask: 0.05 labor, unit in escrow
        [2 * s11 - 2 * s21 - 0.05, 2 * s26 - 8.0],           # trade at the newer order's price (the bid's 10)
        [-0.05, 0.0],                                        # bid of 2: 9 liquid + 2 in escrow = 11
        [0.0, 0.0],                                          # expiry: escrow back to liquid coin
    ])
    assert np.allclose(r, expect, rtol=0, atol=1e-12), (r, expect)


def test_state_along_the_hand_worked_market():
    s, _ = _market_scenario()
    a = s.agents()
    assert list(a["coin64"]) == [11.0, 26.0]
    assert list(a["esc_ticks"]) == [0, 0]
    assert a["inv"].tolist() == [[1, 0], [0, 0]]
    assert list(a["income64"]) == [5.0, 10.0]
    assert a["counts"].tolist() == [[2, 1, 2], [1, 0, 1]]
    assert np.allclose(a["u_prev"], [u_half(11, 3.10), u_half(26, 1.05)], atol=1e-12)


@pytest.mark.parametrize("omega", [1.0, 0.5, 0.0])
def test_government_reward_hand_worked(omega):
    """Eq. 3-5 (READING of Eq. 4: omega (1 - gini) + 1 - omega) on total coin.
    For two agents gini = |x0 - x1| / (2 (x0 + x1)), so the social welfare is
    (x0 + x1) - omega |x0 - x1| / 2.  Totals: (16, 16) until the craft, (21, 16)
    after it, (11, 26) after the trade, unchanged by the resting bid (coin in
    escrow counts) and by its expiry."""
    _, out = _market_scenario(omega=omega)
    g = np.array([o["grew"] for o in out])
    W = lambda x0, x1: (x0 + x1) - omega * abs(x0 - x1) / 2.0
    expect = [0.0, 0.0, W(21, 16) - W(16, 16), W(11, 26) - W(21, 16), 0.0, 0.0]
    assert np.allclose(g, expect, rtol=0, atol=1e-12), (g, expect)


def test_government_reward_of_a_tax_period():
    """Section 3's worked tax example through the environment (three agents):
    agent 0 earns 130, pays 35 at the period end, and each agent receives
    35 / 3.  Totals go from (145, 15, 15) to (110, 15, 15) + 35 / 3; with
    omega = 1 the social welfare is sum - sum_ij |xi - xj| / (2 n), so the
    step's government reward is (260 - 190) / 3."""
    s = Scenario(3, sg=[[2.0, 2.0], [1.0, 1.0], [1.0, 1.0]], sc=[13.0, 0.5, 0.5], T_tax=10,
                 thresholds=[50.0, 100.0], tax_levels=21)
    s.step([gather(0), NOOP, NOOP], gov=[2, 6, 10])          # rates 10 %, 30 %, 50 %
    s.step([gather(1), NOOP, NOOP])
    s.step([craft(), NOOP, NOOP])                            # +130 coin, +130 earnings
    for _ in range(6):
        s.step([NOOP, NOOP, NOOP])
    last = s.step([NOOP, NOOP, NOOP])                        # t = 9: period end
    a = s.agents()
    share = 35.0 / 3.0
    assert a["coin64"] == pytest.approx([145.0 - 35.0 + share, 15.0 + share, 15.0 + share], abs=1e-12)

    def welfare(x):                                          # omega = 1: sum (1 - gini)
        n = len(x)
        pair = sum(abs(xi - xj) for xi in x for xj in x)
        return sum(x) - pair / (2.0 * n)
    before = welfare([145.0, 15.0, 15.0])                    # 175 - 2*2*130/6 = 175 - 86.67
    after = welfare([110.0 + share, 15.0 + share, 15.0 + share])
    assert before == pytest.approx(175.0 - 260.0 / 3.0)
    assert after == pytest.approx(175.0 - 190.0 / 3.0)
    assert last["grew"] == pytest.approx(70.0 / 3.0, abs=1e-9)
    # the population rewards of that step: utility of the new coin, labor unchanged
    eta = 0.27
    u = lambda C: (C ** (1 - eta) - 1) / (1 - eta)
    assert last["rew"] == pytest.approx([u(110 + share) - u(145), u(15 + share) - u(15),
                                         u(15 + share) - u(15)], abs=1e-9)


def test_market_observation_features():
    """App. A market statistics per resource: best bid, best ask (0 when the
    side is empty), resting bids / A and asks / A.  After t2 agent 1's ask of
    6 rests on resource 0; after t4 agent 0's bid of 2 rests on resource 1."""
    s = Scenario(2, sg=[[1.0, 1.0], [1.0, 1.0]], sc=[0.5, 0.25], eta=0.5, start_coin=16.0,
                 Rk=1, Rd=2, gov_enabled=0, expire=2)
    s.step([gather(0), NOOP])
    s.step([gather(1), gather(0)])
    o = s.step([craft(), sell(0, 2)])["obs"]
    for i in range(2):
        assert list(o[i, MKT:MKT + 8]) == [0.0, 6.0, 0.0, 0.5, 0.0, 0.0, 0.0, 0.0]
    s.step([buy(0, 4), NOOP])
    o = s.step([buy(1, 0), NOOP])["obs"]
    for i in range(2):
        assert list(o[i, MKT:MKT + 8]) == [0.0, 0.0, 0.0, 0.0, 2.0, 0.0, 0.5, 0.0]
    # the agent's own columns after t4 (state at t = 5, tax period 100, episode 1000)
    assert o[0, COIN] == 9.0 and o[0, ESC] == 2.0 and o[0, LABOR] == pytest.approx(3.10, abs=1e-12)
    assert list(o[0, INV0:INVE1 + 1]) == [1.0, 0.0, 0.0, 0.0]
    assert list(o[0, SG0:SC + 1]) == [1.0, 1.0, 0.5]
    assert o[0, NORD] == pytest.approx(1.0 / 15.0, abs=1e-15)
    assert o[0, INCOME] == 5.0 and o[1, INCOME] == 10.0
    assert o[0, PLEFT] == pytest.approx(0.95, abs=1e-15) and o[0, TFRAC] == pytest.approx(0.005, abs=1e-15)
    # the government's coin statistics count the 2 coin in escrow: totals (11, 26)
    g = s.env.observe()[1]
    assert g[G_COIN:G_COIN + 3] == pytest.approx([18.5, 7.5, 18.5], abs=1e-12)
    # both sides present, two price levels on each: bids 4 and 2 below asks 8 and 10
    s2 = Scenario(4, sg=np.ones((4, 2)), sc=[0.5] * 4, start_coin=16.0)
    s2.step([gather(0), gather(0), NOOP, NOOP])
    o = s2.step([sell(0, 4), sell(0, 3), buy(0, 1), buy(0, 0)])["obs"]
    assert list(o[2, MKT:MKT + 4]) == pytest.approx([4.0, 8.0, 0.5, 0.5])


def test_government_statistics_odd_population():
    """Fig. 1 caption: mean, standard deviation (population form) and median.
    Three agents craft with skills 0.5, 0.25 and 1.5: coin 21, 18.5, 31 and
    earnings 5, 2.5, 15; labor 3, 3, 3 after gather, gather, craft."""
    s = Scenario(3, sg=np.ones((3, 2)), sc=[0.5, 0.25, 1.5], Rk=1, Rd=2, start_coin=16.0)
    s.step([gather(0)] * 3)
    s.step([gather(1)] * 3)
    g = s.step([craft()] * 3)["gobs"]
    std = math.sqrt((2.5 ** 2 + 5.0 ** 2 + 7.5 ** 2) / 3.0)
    assert g[G_COIN:G_COIN + 3] == pytest.approx([23.5, std, 21.0], abs=1e-12)
    assert g[G_INC:G_INC + 3] == pytest.approx([7.5, std, 5.0], abs=1e-12)
    assert g[G_LAB:G_LAB + 3] == pytest.approx([3.0, 0.0, 3.0], abs=1e-12)


def test_government_statistics_even_population():
    """Four agents with labor 3, 1, 0, 0: mean 1, population std sqrt(6/4),
    median (0 + 1) / 2 = 0.5 (the mean of the two middle values)."""
    s = Scenario(4, sg=np.ones((4, 2)), sc=[0.5] * 4)
    s.step([gather(0), gather(0), NOOP, NOOP])
    s.step([gather(0), NOOP, NOOP, NOOP])
    g = s.step([gather(1), NOOP, NOOP, NOOP])["gobs"]
    assert g[G_LAB:G_LAB + 3] == pytest.approx([1.0, math.sqrt(1.5), 0.5], abs=1e-12)
    assert g[G_COIN:G_COIN + 3] == pytest.approx([15.0, 0.0, 15.0], abs=1e-12)


def test_time_features():
    """Fraction of the tax period left and t / T_ep, for the state after a step
    (T_ep = 20, T_tax = 5): t = 0 -> (1, 0); t = T_tax - 1 = 4 -> (1/5, 4/20);
    t = T_ep - 1 = 19 -> (1/5, 19/20); the step that ends the episode restarts
    it, so its observation is of t = 0 again."""
    s = Scenario(2, T_ep=20, T_tax=5)
    obs, gobs, _ = s.env.observe()
    assert (obs[0, PLEFT], obs[0, TFRAC]) == (1.0, 0.0)
    seen = {}
    for t in range(20):
        r = s.step([NOOP, NOOP])
        seen[t + 1] = (r["obs"][1, PLEFT], r["obs"][1, TFRAC], r["gobs"][G_PLEFT], r["gobs"][G_TFRAC], r["done"])
    assert seen[4][:4] == pytest.approx((0.2, 0.2, 0.2, 0.2))
    assert seen[5][:4] == pytest.approx((1.0, 0.25, 1.0, 0.25))
    assert seen[19][:4] == pytest.approx((0.2, 0.95, 0.2, 0.95))
    assert seen[20] == (1.0, 0.0, 1.0, 0.0, 1)
    assert all(seen[k][4] == 0 for k in range(1, 20))
