"""Host bookkeeping of the trainer's episode measurements (no GPU): returns,
social welfare from the government rewards, productivity and equality, tax
rates at period starts, across rollouts that split an episode."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _buf(T, E, A, nb, rew, grew, done, gobs0, gact):
    return dict(rew=torch.tensor(rew, dtype=torch.float32), grew=torch.tensor(grew, dtype=torch.float32),
                done=torch.tensor(done, dtype=torch.uint8),
                gobs=torch.tensor(gobs0, dtype=torch.float32)[:, :, None].repeat(1, 1, 14),
                gact=torch.tensor(gact, dtype=torch.int32))


def test_episode_log_over_two_rollouts():
    from paper_2410_22165_gb300.train import EpisodeLog
    E, A, nb, T = 2, 3, 3, 4
    log = EpisodeLog(E, A, start_coin=15.0, T_tax=2)
    # episode of 6 steps split over rollouts of 4 and 4 steps (ends at step 5 of the run)
    rew1 = np.ones((T, E, A)); rew1[:, 1, :] = [1.0, 2.0, 6.0]
    grew1 = np.full((T, E), 0.5)
    gobs1 = np.full((T + 1, E), 20.0)
    gact1 = np.arange(T * E * nb).reshape(T, E, nb) % 21
    log.add(0, _buf(T, E, A, nb, rew1, grew1, np.zeros((T, E)), gobs1, gact1))
    assert not log.episodes
    rew2 = np.ones((T, E, A))
    done2 = np.zeros((T, E)); done2[1, :] = 1
    gobs2 = np.full((T + 1, E), 20.0); gobs2[1, 0] = 30.0
    log.add(1, _buf(T, E, A, nb, rew2, grew1, done2, gobs2, gact1))
    assert len(log.episodes) == 2
    e0, e1 = log.episodes
    assert e0["mean_return"] == pytest.approx(6.0) and e0["median_return"] == pytest.approx(6.0)
    # environment 1: rewards 1, 2, 6 per step for 4 steps, then 1 for 2 steps: returns 6, 10, 26
    assert e1["mean_return"] == pytest.approx(14.0) and e1["median_return"] == pytest.approx(10.0)
    # welfare = start coin x A + sum of the episode's government rewards; productivity = A x mean coin
    assert e0["welfare"] == pytest.approx(15.0 * A + 6 * 0.5)
    assert e0["productivity"] == pytest.approx(30.0 * A)
    assert e0["equality"] == pytest.approx((15.0 * A + 3.0) / (30.0 * A))
    # the next episode starts from zero sums; rates recorded every T_tax steps of the episode
    assert np.allclose(log.ret, 2.0) and np.allclose(log.gsum, 1.0)
    assert len(log.rates) == 4           # episode steps 0, 2, 4, then 0 of the next episode
