"""Benchmark of the EconoJax hot path on GB300.

Workload (the env_step throughput configuration): E = 1024 environments x
A = 100 population agents + 1 government, 2 resources, 1000-step episodes,
tax period 100, uniform random seeded actions.  One benchmark step = one
whole episode: env_step with n_steps = 1000 in one launch, inputs (actions,
gather draws, tie-break keys, rate levels; 1.2 GB) resident in HBM, every
output written (rewards, done flags, observations, government observations,
masks; 11 GB).  Inputs and outputs are far larger than L2, so no flush.

Metric: population agent-steps per second (E * A * 1000 per benchmark step).

--impl reference times the CPU oracle (the plain C statement of the rules,
test infrastructure) on the host cores on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "agent-steps/sec (env_step and full rollout) on 1 GB300; PPO updates/sec BF16 vs FP32"
UNIT = "agent-steps/s"
# DRAM bytes (read + write) of the environment kernel measured with ncu on the
# 100-step profile case (E = 1024, A = 100: 129.35 MB read, 1059.60 MB written);
# traffic grows with the steps of a launch (state load/store is once per launch
# and small), so a launch of n steps is reported as n/100 times this.  It
# belongs to the kernel version it was taken on (env_kernel<128, 2, 5> version
# 4.1, 6.00 k warp instructions per environment-step) and is re-taken when that
# changes.
ENV_DRAM_BYTES_PER_100_STEPS = 129354752 + 1059601664
E, A, T_EP, T_TAX = 1024, 100, 1000, 100
CONFIG = {"workload": "env_step E=1024 x A=100 (+1 government), R=2, P=5, 1000-step episode, "
                      "tax period 100, uniform random seeded actions; one benchmark step = one episode "
                      "in one launch",
          "E": E, "A": A, "episode": T_EP, "tax_period": T_TAX,
          "l2": "inputs (1.2 GB) and outputs (11 GB) per step far larger than L2; no flush"}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _bf16_peaks():
    """(burst, sustained) dense BF16 TFLOP/s of MEASURED_PEAKS.json, else the fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", d["bf16_tflops"]))
    except Exception:
        return 1900.0, 1700.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes_per_launch(sizes, n_steps, state_bytes):
    """Bytes env_step must move per launch: streamed inputs and outputs per
    agent-step and per environment-step, plus one load and one store of the
    state per launch."""
    D, G, W = sizes.obs_dim, sizes.gobs_dim, sizes.mask_words
    per_agent_step = 4 + 4 + 4 + 4 + 4 * D + 4 * W           # act, gather u, tie-break key, reward, obs, mask
    per_env_step = 4 + 1 + 4 * G                              # government reward, done, government obs
    gov_in = (n_steps // T_TAX) * 3 * 4                       # rate levels read at period starts
    return n_steps * E * (A * per_agent_step + per_env_step) + E * gov_in + 2 * state_bytes


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2410_22165_gb300 import VecEnv
    from paper_2410_22165_gb300 import build as cuda_build

    rank, world, local = _dist()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0:
        cuda_build.build()
    if world > 1:
        dist.barrier()

    seed = 1000 + rank                     # replicas: each rank runs its own environments
    env = VecEnv(E, A, device=dev, T_ep=T_EP, T_tax=T_TAX)
    env.reset(seed=seed)
    d = env.fill_draws(seed=seed, g0=0, n_steps=T_EP)
    out = env.alloc_outputs(T_EP)
    stream = torch.cuda.current_stream(dev)

    def one_step():
        env.step(T_EP, act=d["act"], gov_act=d["gov_act"], gather_u=d["gather_u"], tb=d["tb"], out=out)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        time.sleep(0.4)
        torch.cuda.synchronize(dev)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            starts[k].record(stream)
            one_step()
            ends[k].record(stream)
        t1.record(stream)
        torch.cuda.synchronize(dev)
    total_ms = t0.elapsed_time(t1)
    launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
        dist.barrier()

    agent_steps = E * A * T_EP * args.steps * world
    value = agent_steps / (total_ms / 1e3)

    # end to end through the public API: pinned host inputs -> device, episode, outputs -> host
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(env, d, out, args, dev, world)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    peak, peak_kind = _peaks()
    bytes_launch = algorithmic_bytes_per_launch(env.sizes, T_EP, env.sizes.state_bytes)
    avg_launch_s = statistics.mean(launch_ms) / 1e3
    achieved = bytes_launch / avg_launch_s / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32",
        "data": "synthetic (Philox-4x32-10 seeded draws)", "config": dict(CONFIG, replicas=world),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                     "traffic": ENV_DRAM_BYTES_PER_100_STEPS * T_EP / 100,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the 100-step profile "
                                       "case, scaled to the launch's steps",
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "kernel": "env_kernel<128>", "launch_ms": statistics.mean(launch_ms)},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_train:
        del d, out
        torch.cuda.empty_cache()
        line["single_step"] = run_single_step(args, dev)
        line["rollout"] = {"workload": "E=4096 x A=100, 1000 steps: policy + sampling + government policy + "
                                       "env_step per step",
                           "bf16": run_rollout(args, dev, "bf16"), "fp32": run_rollout(args, dev, "fp32")}
        line["ppo"] = {"workload": "E=2048 x A=100 x 128 steps, GAE, 4 epochs x 8 minibatches, both networks",
                       "bf16": run_ppo(args, dev, "bf16"), "fp32": run_ppo(args, dev, "fp32")}
        line["batched"] = run_batched(args, dev)
        line["section5"] = run_section5(args, dev)
        if args.train_updates > 0 and world == 1:
            line["training"] = run_training(args, dev)
        line["multi_agent"] = run_multi_agent(args, dev)
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if world > 1:
        dist.destroy_process_group()
    return line


def run_single_step(args, dev, seed=1000):
    """env_step in single-step mode: the headline workload (E x A, one
    1000-step episode, every output) with one launch per step, so that the
    state goes through HBM every step; the 1000 launches are one CUDA graph.
    Algorithmic bytes per launch: the step's inputs and outputs plus one load
    and one store of the state without the order book (whose live part
    varies; leaving it out keeps the figure a lower bound)."""
    import torch

    from paper_2410_22165_gb300 import VecEnv
    from paper_2410_22165_gb300 import _native as N

    env = VecEnv(E, A, device=dev, T_ep=T_EP, T_tax=T_TAX)
    env.reset(seed=seed)
    d = env.fill_draws(seed=seed, g0=0, n_steps=T_EP)
    out = env.alloc_outputs(T_EP)

    def episode(stream=None):
        for t in range(T_EP):
            env.step(1, act=d["act"][t:t + 1], gov_act=d["gov_act"][t:t + 1], gather_u=d["gather_u"][t:t + 1],
                     tb=d["tb"][t:t + 1], out={k: v[t:t + 1] for k, v in out.items()}, stream=stream)

    episode()
    torch.cuda.synchronize(dev)
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            episode(stream=s)
    torch.cuda.current_stream(dev).wait_stream(s)
    g.replay()
    torch.cuda.synchronize(dev)
    steps = max(1, min(args.steps, 3))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        g.replay()
    b.record()
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    off, cnt, esz = N.state_field(env.p, "book")
    state_wo_book = env.sizes.state_bytes - cnt * esz
    per_launch = algorithmic_bytes_per_launch(env.sizes, 1, state_wo_book)
    peak, kind = _peaks()
    achieved = per_launch * T_EP / (ms / 1e3) / 1e9
    out_d = {"workload": f"env_step E={E} x A={A}, one launch per step over a {T_EP}-step episode (one CUDA graph)",
             "value": E * A * T_EP / (ms / 1e3), "unit": UNIT, "ms_per_episode": ms, "launches_per_episode": T_EP,
             "algorithmic_bytes_per_launch": per_launch, "achieved_GBps": achieved, "frac_of_hbm": achieved / peak,
             "peak_source": f"{kind} hbm_gbs"}
    del g, out, d, env
    torch.cuda.empty_cache()
    return out_d


def run_rollout(args, dev, precision, E_r=4096, T_r=1000, seed=2000):
    """Full rollout: E_r x A policy forward + masked sampling + government
    policy + env_step per step, T_r steps (BF16: the two networks share one
    launch, 2 launches per step; FP32: 3), from 2048 environments in two
    independent chains of environments on two streams."""
    import torch

    import synth
    from paper_2410_22165_gb300 import Policy, Rollout, VecEnv

    env = VecEnv(E_r, A, device=dev, T_ep=T_EP, T_tax=T_TAX)
    pw = torch.from_numpy(synth.net_weights(seed, 0, env.D, 128, env.nA))
    gw = torch.from_numpy(synth.net_weights(seed, 1, env.G, 128, env.p.nb * env.p.tax_levels))
    pol = Policy(env, pw, gw, hidden=128, precision=precision)
    ro = Rollout(env, pol, T_r)
    ro.reset(seed=seed)
    ro.run()
    ro.capture()                    # the whole T_r-step rollout as one CUDA graph
    torch.cuda.synchronize(dev)
    steps = max(1, min(args.steps, 2))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        ro.replay()
    b.record()
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    mean_rew = float(ro.buf["rew"].double().mean().item())
    out = {"value": E_r * A * T_r / (ms / 1e3), "unit": UNIT, "ms_per_rollout": ms,
           "mean_population_reward": mean_rew, "launches_per_rollout": (2 if E_r >= 2048 else 1) * (2 * T_r + 1 if precision == "bf16" else 3 * T_r + 2),
           "chains": 2 if E_r >= 2048 else 1,
           "graph": "one CUDA graph per rollout (carry-over copies + all launches)"}
    del ro, pol, env
    torch.cuda.empty_cache()
    return out


def ppo_flops_per_row(in_dim, H, O):
    """Useful FLOPs of one minibatch row of the PPO gradient: actor and critic
    forward, backward-data through the hidden layers (not into the inputs),
    and the weight gradients (as many multiply-adds as the forward)."""
    fwd = in_dim * H + H * H + H * O + in_dim * H + H * H + H
    bwd_data = O * H + H * H + H * H
    return 2 * (2 * fwd + bwd_data)


def run_ppo(args, dev, precision, E_p=2048, T_p=128, seed=3000):
    """One training iteration of config 4 in the given precision: a T_p-step
    rollout of E_p x A agents (policy, sampling, env_step), then the PPO update
    (GAE, 4 epochs x 8 minibatches of the population and government
    networks).  Reports updates/s and rollout+update agent-steps/s.  With N
    ranks each rank rolls out its own E_p environments and the update is the
    data-parallel one (DistributedPPO: advantage moments and gradients summed
    over the ranks by NCCL all-reduces)."""
    import torch

    import synth
    from paper_2410_22165_gb300 import PPO, Policy, Rollout, VecEnv
    from paper_2410_22165_gb300.distributed import DistributedPPO

    rank, world, _ = _dist()

    env = VecEnv(E_p, A, device=dev, T_ep=T_EP, T_tax=T_TAX)
    pw = torch.from_numpy(synth.net_weights(seed, 0, env.D, 128, env.nA))
    gw = torch.from_numpy(synth.net_weights(seed, 1, env.G, 128, env.p.nb * env.p.tax_levels))
    pol = Policy(env, pw, gw, hidden=128, precision=precision)
    ro = Rollout(env, pol, T_p)
    ro.reset(seed=seed + rank)
    ro.run()
    ppo = PPO(pol, T_p, precision=precision)
    update = DistributedPPO(ppo).update if world > 1 else ppo.update
    update(ro)
    torch.cuda.synchronize(dev)
    steps = max(1, min(args.steps, 2))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ms = ro_ms = 0.0
    for _ in range(steps):
        ev[0].record()
        ro.carry_over()
        ro.run()
        ev[1].record()
        stats = update(ro)
        ev[2].record()
        torch.cuda.synchronize(dev)
        ro_ms += ev[0].elapsed_time(ev[1]) / steps
        ms += ev[1].elapsed_time(ev[2]) / steps
    if world > 1:   # sums over ranks and minibatches -> means over all rows of the update
        n_rows = torch.tensor([[E_p * A], [E_p]], dtype=torch.float64, device=stats.device)
        stats = (stats[:, 2:5] / (n_rows * T_p * ppo.pp.epochs * world)).float()
    st = stats.cpu().numpy()
    rows = ppo.pp.epochs * T_p * E_p * world
    flops = rows * (A * ppo_flops_per_row(env.D, 128, env.nA) + ppo_flops_per_row(env.G, 128, env.p.nb * env.p.tax_levels))
    out = {"updates_per_s": 1e3 / ms, "ms_per_update": ms, "precision": precision,
           "rollout_ms": ro_ms, "train_agent_steps_per_s": world * E_p * A * T_p / ((ro_ms + ms) / 1e3),
           "useful_TFLOPs": flops / (ms / 1e3) / 1e12, "useful_TFLOP_per_update": flops / 1e12,
           "peak_TFLOPs": (_bf16_peaks()[1] if precision == "bf16" else FP32_FMA_TFLOPS),
           "peak_source": ("measured bf16_tflops_sustained" if precision == "bf16" else
                           "derived FP32 FMA peak: 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz"),
           "transitions_per_update": world * E_p * A * T_p, "epochs": ppo.pp.epochs, "minibatches": ppo.pp.minibatches,
           "ranks": world,
           "population_loss": {"policy": float(st[0, 0]), "value": float(st[0, 1]), "entropy": float(st[0, 2])}}
    out["frac_of_peak"] = out["useful_TFLOPs"] / out["peak_TFLOPs"]
    del ppo, ro, pol, env
    torch.cuda.empty_cache()
    return out


FP32_FMA_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # derived: SMs x FP32 lanes x 2 FLOP x max SM clock


def run_training(args, dev, E_t=2048, T_t=128, seed=3000):
    """Learning behaviour of the two precisions (Section 4's simultaneous
    training of the population and government networks): `--train-updates`
    iterations of {T_t-step rollout, PPO update} of E_t x A agents, in BF16
    and in FP32, from the same initial weights and environment seed.
    Returns per iteration the mean population reward per agent-step and the
    mean government reward per environment-step, and the mean episodic
    returns (sum over an episode's steps; population: averaged over the
    agents) of the episodes completed in the last third of the run, with the
    standard error over environments.  The two runs sample different actions
    as soon as their policies differ, so they agree statistically, not bit
    for bit; a third run (BF16, the next seed) gives the difference that the
    seed alone makes, the scale against which the precision's is read."""
    import numpy as np
    import torch

    import synth
    from paper_2410_22165_gb300 import PPO, Policy, Rollout, VecEnv

    n_up = args.train_updates
    out = {"workload": f"E={E_t} x A={A}, {n_up} iterations of a {T_t}-step rollout + PPO update "
                       "(4 epochs x 8 minibatches), both networks, same seed for both precisions"}
    for run, precision, sd in (("bf16", "bf16", seed), ("fp32", "fp32", seed), ("bf16_seed2", "bf16", seed + 1)):
        env = VecEnv(E_t, A, device=dev, T_ep=T_EP, T_tax=T_TAX)
        pw = torch.from_numpy(synth.net_weights(sd, 0, env.D, 128, env.nA))
        gw = torch.from_numpy(synth.net_weights(sd, 1, env.G, 128, env.p.nb * env.p.tax_levels))
        pol = Policy(env, pw, gw, hidden=128, precision=precision)
        ro = Rollout(env, pol, T_t)
        ro.reset(seed=sd)
        ppo = PPO(pol, T_t, precision=precision)
        ep_pop = np.zeros(E_t)
        ep_gov = np.zeros(E_t)
        finished = []                    # (iteration, population return, government return) per episode
        curve_pop, curve_gov = [], []
        t0 = time.perf_counter()
        for it in range(n_up):
            if it:
                ro.carry_over()
            ro.run()
            rew = ro.buf["rew"].double().mean(dim=2).cpu().numpy()      # [T, E]
            grew = ro.buf["grew"].double().cpu().numpy()
            done = ro.buf["done"].cpu().numpy()
            curve_pop.append(float(rew.mean()))
            curve_gov.append(float(grew.mean()))
            for t in range(T_t):
                ep_pop += rew[t]
                ep_gov += grew[t]
                for e in np.nonzero(done[t])[0]:
                    finished.append((it, ep_pop[e], ep_gov[e]))
                ep_pop[done[t] != 0] = 0.0
                ep_gov[done[t] != 0] = 0.0
            ppo.update(ro)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        late = [f for f in finished if f[0] >= (2 * n_up) // 3] or finished
        rp = np.array([f[1] for f in late]) if late else np.zeros(1)
        rg = np.array([f[2] for f in late]) if late else np.zeros(1)
        out[run] = {
            "mean_population_reward_per_iteration": curve_pop, "mean_government_reward_per_iteration": curve_gov,
            "episodes_completed": len(finished), "late_episodes": len(late),
            "late_population_return": float(rp.mean()), "late_population_return_se": float(rp.std() / np.sqrt(len(rp))),
            "late_government_return": float(rg.mean()), "late_government_return_se": float(rg.std() / np.sqrt(len(rg))),
            "wall_s": wall}
        del ppo, ro, pol, env
        torch.cuda.empty_cache()
    b, f, b2 = out["bf16"], out["fp32"], out["bf16_seed2"]
    for who in ("population", "government"):
        key, se = f"late_{who}_return", f"late_{who}_return_se"
        # precision effect (same seed) next to the seed effect (same precision)
        out[f"{who}_return_difference"] = b[key] - f[key]
        out[f"{who}_return_difference_se"] = float(np.hypot(b[se], f[se]))
        out[f"{who}_return_seed_difference"] = b[key] - b2[key]
        out[f"{who}_return_seed_difference_se"] = float(np.hypot(b[se], b2[se]))
    return out


def run_paper_training(args, dev):
    """Section 4's experiment at Table 2's settings: the population and the
    government trained simultaneously for 1e7 environment steps (rollouts of
    150 steps in 10 environments, 6 epochs x 6 minibatches, gamma 0.999,
    learning rate 5e-4 and entropy coefficient 0.1 annealed), once with taxes
    and once as a free market (no government), from the same seed.  Prints
    the episode measurements of the first and the last tenth of the run."""
    import torch

    import synth
    from paper_2410_22165_gb300 import Policy, VecEnv
    from paper_2410_22165_gb300.train import Trainer

    E_t, T_t = args.paper_envs, 150
    skills = {"uniform": 0, "normal": 1}[args.paper_skills]
    th = [float(x) for x in args.paper_thresholds.split(",")]
    iters = int(round(args.paper_env_steps / (E_t * T_t)))
    out = {"workload": f"Section 4 training: {E_t} environments x {A} agents, rollouts of {T_t} steps, "
                       f"{iters} iterations = {iters * E_t * T_t:.3g} environment steps, 6 epochs x 6 minibatches, "
                       "gamma 0.999, lr 5e-4 and entropy 0.1 annealed (Table 2), BF16, skills "
                       + ("U[0,1)" if skills == 0 else "around 1 with sd 1 (Section 5's reading)")
                       + f", bracket edges {th}",
           "precision": "bf16"}
    for label, taxes in (("taxes", True), ("free_market", False)):
        env = VecEnv(E_t, A, device=dev, T_ep=T_EP, T_tax=T_TAX, gov_enabled=1 if taxes else 0, skill_init=skills,
                     thresholds=th)
        pw = torch.from_numpy(synth.net_weights(args.paper_seed, 0, env.D, 128, env.nA))
        gw = torch.from_numpy(synth.net_weights(args.paper_seed, 1, env.G, 128, env.p.nb * env.p.tax_levels))
        pol = Policy(env, pw, gw, hidden=128, precision="bf16")
        tr = Trainer(pol, T=T_t, precision="bf16", total_iterations=iters, seed=args.paper_seed, gamma=0.999,
                     epochs=6, minibatches=6)
        tr.reset(seed=args.paper_seed)
        wall = tr.train()
        out[label] = dict(tr.summary(), wall_s=wall,
                          agent_steps_per_s=iters * E_t * T_t * A / wall)
        del tr, pol, env
        torch.cuda.empty_cache()
    return out


def run_multi_agent(args, dev, E_m=256, T_m=32, H_m=256, seed=6000):
    """Section 5's three multi-agent methods on its 4-resource market (30
    actions, prices 3, 6, 9, no taxes, skills around 1 growing by 0.5 %,
    networks of 256 units), float32: one training iteration (a T_m-step
    rollout of E_m x A agents, then a PPO update, 4 epochs x 8 minibatches)
    with the population's networks shared, independent (an actor and a critic
    per agent) and CTDE (an actor per agent, one critic); and the rollout
    again with the BF16 forward (the update at hidden 256 is float32)."""
    import numpy as np
    import torch

    import synth
    from paper_2410_22165_gb300 import PPO, Policy, Rollout, VecEnv

    out = {"workload": f"Section 5: E={E_m} x A={A}, R=4 (30 actions), no taxes, skills around 1 growing, "
                       f"hidden {H_m}, FP32, {T_m}-step rollout + PPO update (4 epochs x 8 minibatches)"}
    kw = dict(R=4, P=3, price_ticks=[1, 2, 3], price_tick=3.0, Rd=2, gov_enabled=0, skill_gain=0.005,
              skill_init=1, T_ep=T_EP, T_tax=T_TAX)
    env = VecEnv(E_m, A, device=dev, **kw)
    shared = synth.net_weights(seed, 0, env.D, H_m, env.nA)
    per_agent = np.concatenate([synth.net_weights(seed, 10 + i, env.D, H_m, env.nA) for i in range(A)])
    gw = torch.from_numpy(synth.net_weights(seed, 1, env.G, H_m, env.p.nb * env.p.tax_levels))
    del env
    for layout in ("shared", "independent", "ctde"):
        env = VecEnv(E_m, A, device=dev, **kw)
        pw = torch.from_numpy(shared if layout == "shared" else per_agent)
        pol = Policy(env, pw, gw, hidden=H_m, precision="fp32", layout=layout)
        ro = Rollout(env, pol, T_m)
        ro.reset(seed=seed)
        ro.run()
        ppo = PPO(pol, T_m, precision="fp32")
        ppo.update(ro)
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        ro.carry_over()
        ro.run()
        ev[1].record()
        ppo.update(ro)
        ev[2].record()
        torch.cuda.synchronize(dev)
        ro_ms, up_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        # the same rollout with the BF16 forward (hidden 256: the two-CTA cluster kernel)
        pol16 = Policy(env, pw, gw, hidden=H_m, precision="bf16", layout=layout)
        ro16 = Rollout(env, pol16, T_m)
        ro16.reset(seed=seed)
        ro16.run()
        torch.cuda.synchronize(dev)
        ev[0].record()
        ro16.carry_over()
        ro16.run()
        ev[1].record()
        torch.cuda.synchronize(dev)
        ro16_ms = ev[0].elapsed_time(ev[1])
        out[layout] = {"rollout_ms": ro_ms, "update_ms": up_ms, "population_parameters": int(pw.numel()),
                       "train_agent_steps_per_s": E_m * A * T_m / ((ro_ms + up_ms) / 1e3),
                       "rollout_ms_bf16": ro16_ms,
                       "rollout_agent_steps_per_s": {"fp32": E_m * A * T_m / (ro_ms / 1e3),
                                                     "bf16": E_m * A * T_m / (ro16_ms / 1e3)}}
        del ppo, ro, pol, ro16, pol16, env
        torch.cuda.empty_cache()
    return out


def run_section5(args, dev, E_s=1024, T_s=1000, seed=5000):
    """Section 5's multi-resource environments (no taxes, prices 3, 6, 9,
    skills around 1 that grow by 0.5 % per gather / craft, R_d = log2 R):
    env_step of E_s x A agents over one T_s-step episode in one launch, with
    the draws made in the kernel, at 4 and 12 resources."""
    import torch

    from paper_2410_22165_gb300 import VecEnv

    out = {}
    for R, Rd in ((4, 2), (12, 3)):
        env = VecEnv(E_s, A, device=dev, T_ep=T_s, T_tax=T_TAX, R=R, P=3, price_tick=3.0, price_ticks=[1, 2, 3],
                     Rd=Rd, gov_enabled=0, skill_gain=0.005, skill_init=1)
        env.reset(seed=seed)
        o = env.alloc_outputs(T_s)
        env.step(T_s, out=o)                      # warm-up episode
        torch.cuda.synchronize(dev)
        ms = []
        for _ in range(max(1, min(args.steps, 3))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            env.step(T_s, out=o)
            b.record()
            torch.cuda.synchronize(dev)
            ms.append(a.elapsed_time(b))
        m = statistics.median(ms)
        out[f"R{R}"] = {"value": E_s * A * T_s / (m / 1e3), "unit": UNIT, "ms_per_episode": m,
                        "actions": env.nA, "mean_skill_end": float(env.field("sg")[:, :, :A].float().mean().item())}
        del env, o
        torch.cuda.empty_cache()
    out["workload"] = (f"E={E_s} x A={A}, {T_s}-step episode in one launch, draws in the kernel; R resources, "
                       "prices 3/6/9, no taxes, skill growth 0.5 % to a maximum of 5, skills around 1")
    return out


def run_batched(args, dev, E_b=2048, T_b=1000, seed=4000):
    """Config 5: E_b environments with populations drawn uniformly from
    {10, 50, 100, 250, 500} and price grids from {5, 10, 20} levels (24, 44,
    84 actions), one network per action-space size; the partition into
    classes is chosen by the autotuner (64-step probes: long enough that the
    replay's fixed costs, such as the per-class slot-0 copies, do not decide), then one T_b-step
    rollout of all classes is one CUDA-graph replay, timed with events."""
    import numpy as np
    import torch

    import synth
    from paper_2410_22165_gb300 import BatchedRollout, VecEnv, autotune, price_grid

    rng = np.random.default_rng(seed)
    pops = rng.choice([10, 50, 100, 250, 500], E_b).tolist()
    levels = rng.choice([5, 10, 20], E_b).tolist()
    weights = {}
    for P in (5, 10, 20):
        probe = VecEnv(1, 10, device=dev, **price_grid(P))
        weights[("pop", P)] = torch.from_numpy(synth.net_weights(seed + P, 0, probe.D, 128, probe.nA))
        weights[("gov",)] = torch.from_numpy(synth.net_weights(seed, 1, probe.G, 128,
                                                               probe.p.nb * probe.p.tax_levels))
        del probe
    kw = dict(T_ep=T_EP, T_tax=T_TAX)
    from paper_2410_22165_gb300.batch import parse_candidate
    best, rates = autotune(pops, levels, weights, T_probe=64, repeats=5, device=dev,
                           candidates=("exact", "pow2", "coarse", "exact+merge", "coarse+merge", "exact+merge+chains2",
                                       "exact+chains1", "exact+chains2", "pow2+chains2"), **kw)
    gran, merged, chains = parse_candidate(best)
    br = BatchedRollout(pops, levels, T_b, weights, granularity=gran, merge=merged, chains=chains, device=dev, **kw)
    br.reset(seed=seed)
    br.capture()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    br.run()
    b.record()
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b)
    out = {"workload": f"E={E_b} environments, populations from {{10,50,100,250,500}} ({sum(pops)} agents), "
                       f"price grids from {{5,10,20}} levels, {T_b} steps, BF16 policy, one graph replay",
           "value": br.agent_steps / (ms / 1e3), "unit": UNIT, "ms_per_rollout": ms, "partition": best,
           "classes": len(br.classes), "autotune_agent_steps_per_s": rates}
    del br
    torch.cuda.empty_cache()
    return out


def run_e2e(env, d, out, args, dev, world):
    """Same metric through the C ABI's host-buffer call env_step_host (via
    VecEnv.step_host, argument marshalling only): each step's inputs come
    from pinned host memory and all its outputs go back to it, in 100-step
    chunks whose copies the library overlaps with the kernel of the next."""
    import torch

    chunk = 100
    host_in = {k: v.cpu().pin_memory() for k, v in d.items()}
    host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
    h2d = sum(v.numel() * v.element_size() for v in host_in.values())
    d2h = sum(v.numel() * v.element_size() for v in host_out.values())

    def one():
        env.step_host(T_EP, host_in, host_out, chunk=chunk, sync=False)

    steps = max(3, min(args.steps, 5))
    one()
    torch.cuda.synchronize(dev)
    # each episode timed on its own (host clock around enqueue + completion); the host link is shared
    # with the machine's other jobs, so the median episode is reported, with every episode's rate
    secs = []
    for _ in range(steps):
        t0 = time.perf_counter()
        one()
        torch.cuda.synchronize(dev)
        secs.append(time.perf_counter() - t0)
    dt = sorted(secs)[len(secs) // 2]
    return {"value": E * A * T_EP * world / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps, "statistic": "median episode",
            "episode_rates": [E * A * T_EP * world / s for s in secs],
            "link_GBps": (h2d + d2h) / dt / 1e9,
            "how": "C ABI env_step_host, 100-step chunks: pinned host inputs copied in and all outputs copied "
                   "out by the library, copies of one chunk overlapping the kernel of the next"}


# ------------------------------------------------------------- CPU oracle

def _oracle_episode(e, seed, n_steps):
    import synth
    from oracle.env import OracleEnv, default_params

    p = default_params(T_ep=T_EP, T_tax=T_TAX)
    o = OracleEnv(p, A)
    inp = synth.episode_inputs(seed, [e], A, p["R"], p["nb"], o.nA, p["tax_levels"], n_steps, p["T_ep"])
    o.reset(inp["sg0"][0], inp["sc0"][0])
    t0 = time.perf_counter()
    o.run(inp["act"][:, 0], inp["gov_act"][:, 0], inp["gather_u"][:, 0], inp["tb"][:, 0],
          inp["later_sg"][:, 0], inp["later_sc"][:, 0], outputs=True)
    return time.perf_counter() - t0


def oracle_throughput(target_s: float):
    """Runs whole oracle episodes (A = 100, 1000 steps) on all host cores in
    threads (the C oracle releases the GIL) for about target_s seconds."""
    import concurrent.futures as cf

    from oracle import build as oracle_build

    oracle_build.build()
    cores = os.cpu_count() or 1
    probe = _oracle_episode(0, 0, 100)             # seconds per 100 steps of one environment
    per_env = probe * (T_EP / 100)
    n_env = max(cores, int(round(target_s * cores / max(per_env, 1e-3) / cores)) * cores)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda e: _oracle_episode(e, 0, T_EP), range(n_env)))
    wall = time.perf_counter() - t0
    value = n_env * A * T_EP / wall
    sample = f"{n_env} environments x A={A} x {T_EP} steps (whole episodes, all outputs), {wall:.1f} s wall"
    single = A * 100 / probe                       # one thread: the probe's 100 steps of one environment
    return value, cores, sample, single


def cpu_baseline(target_s):
    value, cores, sample, single = oracle_throughput(target_s)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "single_thread": single}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return None
    per_step = []
    for _ in range(args.warmup):
        oracle_throughput(args.ref_seconds)
    for _ in range(args.steps):
        v, cores, sample, _ = oracle_throughput(args.ref_seconds)
        per_step.append(v)
    value = statistics.mean(per_step)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 mirror",
        "data": "synthetic (Philox-4x32-10 seeded draws)", "config": CONFIG,
        "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": value, "unit": UNIT},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_profile_case(args):
    """Small cases for profilers (a few GB on the device at most).
    env: E = 1024 x A = 100, 100-step launches (inputs 123 MB, outputs 1.1 GB).
    policy: population policy forward on E = 4096 x A = 100 rows, bf16 then fp32.
    ppo: one PPO update of E = 256 x A = 100 x 32 steps (8 minibatches)."""
    import torch

    from paper_2410_22165_gb300 import VecEnv

    if args.profile_case == "policy":
        import synth
        from paper_2410_22165_gb300 import Policy
        from paper_2410_22165_gb300 import _native as N
        env = VecEnv(4096, A, device="cuda", T_ep=T_EP, T_tax=T_TAX)
        env.reset(seed=7)
        o = env.step(3)
        obs, mask = o["obs"][-1].contiguous(), o["mask"][-1].contiguous()
        pw = torch.from_numpy(synth.net_weights(7, 0, env.D, 128, env.nA))
        gw = torch.from_numpy(synth.net_weights(7, 1, env.G, 128, env.p.nb * env.p.tax_levels))
        res = {}
        for prec in ("bf16", "fp32"):
            pol = Policy(env, pw, gw, hidden=128, precision=prec)
            ms = []
            for k in range(args.warmup + args.steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                pol.forward(N.NET_POP, obs, mask)
                b.record()
                torch.cuda.synchronize()
                if k >= args.warmup:
                    ms.append(a.elapsed_time(b))
            flops = 4096 * A * 2 * (env.D * 128 * 2 + 128 * 128 * 2 + 128 * env.nA + 128)
            res[prec] = {"launch_ms": ms, "useful_TFLOPs": flops / (statistics.mean(ms) / 1e3) / 1e12}
        print(json.dumps({"profile_case": "policy E=4096 A=100", **res}))
        return
    if args.profile_case == "env1":
        # single-step mode of the headline workload: one launch per step (state
        # through HBM or L2 every step), E = 1024 x A = 100, every output
        env = VecEnv(E, A, device="cuda", T_ep=T_EP, T_tax=T_TAX)
        env.reset(seed=7)
        n = args.warmup + args.steps
        d = env.fill_draws(seed=7, g0=0, n_steps=n)
        out = env.alloc_outputs(n)
        ms = []
        for k in range(n):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            env.step(1, act=d["act"][k:k + 1], gov_act=d["gov_act"][k:k + 1], gather_u=d["gather_u"][k:k + 1],
                     tb=d["tb"][k:k + 1], out={key: v[k:k + 1] for key, v in out.items()})
            b.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                ms.append(a.elapsed_time(b))
        print(json.dumps({"profile_case": "env single-step E=1024 A=100", "launch_ms": ms}))
        return
    if args.profile_case == "policy256":
        # population forward with Section 5's networks of 256 units: the default
        # market (24 actions) and the 4-resource market (46 actions), BF16 and FP32
        import synth
        from paper_2410_22165_gb300 import Policy
        from paper_2410_22165_gb300 import _native as N
        s5 = dict(R=4, Rd=2, P=3, price_tick=3.0, price_ticks=[1, 2, 3], gov_enabled=0, skill_gain=0.005,
                  skill_init=1)
        res = {}
        for label, kw in (("default", {}), ("R4", s5)):
            env = VecEnv(4096, A, device="cuda", T_ep=T_EP, T_tax=T_TAX, **kw)
            env.reset(seed=7)
            o = env.step(3)
            obs, mask = o["obs"][-1].contiguous(), o["mask"][-1].contiguous()
            pw = torch.from_numpy(synth.net_weights(7, 0, env.D, 256, env.nA))
            gw = torch.from_numpy(synth.net_weights(7, 1, env.G, 256, env.p.nb * env.p.tax_levels))
            flops = 4096 * A * 2 * (env.D * 256 * 2 + 256 * 256 * 2 + 256 * env.nA + 256)
            for prec in ("bf16", "fp32"):
                pol = Policy(env, pw, gw, hidden=256, precision=prec)
                ms = []
                for k in range(args.warmup + args.steps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    pol.forward(N.NET_POP, obs, mask)
                    b.record()
                    torch.cuda.synchronize()
                    if k >= args.warmup:
                        ms.append(a.elapsed_time(b))
                res[f"{label}_{prec}"] = {"launch_ms": statistics.median(ms),
                                          "useful_TFLOPs": flops / (statistics.median(ms) / 1e3) / 1e12}
        print(json.dumps({"profile_case": "policy hidden 256, E=4096 A=100", **res}))
        return
    if args.profile_case == "ppo":
        import synth
        from paper_2410_22165_gb300 import PPO, Policy, Rollout
        env = VecEnv(256, A, device="cuda", T_ep=T_EP, T_tax=T_TAX)
        pw = torch.from_numpy(synth.net_weights(7, 0, env.D, 128, env.nA))
        gw = torch.from_numpy(synth.net_weights(7, 1, env.G, 128, env.p.nb * env.p.tax_levels))
        pol = Policy(env, pw, gw, hidden=128, precision="bf16")
        ro = Rollout(env, pol, 32)
        ro.reset(seed=7)
        ro.run()
        res = {}
        for prec in ("bf16", "fp32"):
            ppo = PPO(pol, 32, precision=prec)
            ms = []
            for k in range(args.warmup + args.steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                ppo.update(ro)
                b.record()
                torch.cuda.synchronize()
                if k >= args.warmup:
                    ms.append(a.elapsed_time(b))
            res[prec] = {"update_ms": ms}
        print(json.dumps({"profile_case": "ppo E=256 A=100 T=32", **res}))
        return
    if args.profile_case == "ppo4":
        # the PPO configuration's BF16 update: a 128-step rollout of 2048
        # environments, then timed updates (4 epochs x 8 minibatches)
        import synth
        from paper_2410_22165_gb300 import PPO, Policy, Rollout
        env = VecEnv(2048, A, device="cuda", T_ep=T_EP, T_tax=T_TAX)
        pw = torch.from_numpy(synth.net_weights(7, 0, env.D, 128, env.nA))
        gw = torch.from_numpy(synth.net_weights(7, 1, env.G, 128, env.p.nb * env.p.tax_levels))
        pol = Policy(env, pw, gw, hidden=128, precision="bf16")
        ro = Rollout(env, pol, 128)
        ro.reset(seed=7)
        ro.run()
        ppo = PPO(pol, 128, precision="bf16")
        ms = []
        for k in range(args.warmup + args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ppo.update(ro)
            b.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                ms.append(a.elapsed_time(b))
        print(json.dumps({"profile_case": "ppo E=2048 A=100 T=128 bf16", "update_ms": ms}))
        return

    n = 100
    env = VecEnv(E, A, device="cuda", T_ep=T_EP, T_tax=T_TAX)
    env.reset(seed=7)
    d = env.fill_draws(seed=7, g0=0, n_steps=n)
    out = env.alloc_outputs(n)
    ms = []
    for k in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        env.step(n, act=d["act"], gov_act=d["gov_act"], gather_u=d["gather_u"], tb=d["tb"], out=out)
        b.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            ms.append(a.elapsed_time(b))
    bytes_launch = algorithmic_bytes_per_launch(env.sizes, n, env.sizes.state_bytes)
    print(json.dumps({"profile_case": "E=1024 A=100 n_steps=100", "launch_ms": ms,
                      "algorithmic_bytes_per_launch": bytes_launch,
                      "achieved_GBps": bytes_launch / (statistics.mean(ms) / 1e3) / 1e9}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-case", nargs="?", const="env", default=None, choices=["env", "env1", "policy", "policy256", "ppo", "ppo4"])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-train", action="store_true", help="skip the rollout and PPO measurements")
    ap.add_argument("--train-updates", type=int, default=20,
                    help="iterations of the BF16 / FP32 training comparison (0: skip)")
    ap.add_argument("--paper-training", action="store_true",
                    help="run Section 4's training experiment (taxes vs free market) instead of the benchmark")
    ap.add_argument("--paper-envs", type=int, default=10)
    ap.add_argument("--paper-env-steps", type=float, default=1e7)
    ap.add_argument("--paper-seed", type=int, default=7)
    ap.add_argument("--paper-skills", default="uniform", choices=["uniform", "normal"])
    ap.add_argument("--paper-thresholds", default="50,100",
                    help="tax bracket edges (default: the worked example's; the paper's Dutch 2025 brackets / 100 "
                         "are not printed)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.profile_case:
        run_profile_case(args)
        return
    if args.paper_training:
        import torch
        from paper_2410_22165_gb300 import build as cuda_build
        cuda_build.build()
        print(json.dumps(run_paper_training(args, torch.device("cuda", 0))), flush=True)
        return
    line = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
