"""Batched sweep and continuous-batching serving of gear-bath cases on one GPU.

    python -m paper_2512_09904_b300.serving sweep [--cases 64] [--steps 50] [--count-scale 1.0]
    python -m paper_2512_09904_b300.serving serve [--requests 64] [--steps 200] [--rate 4] ...
    torchrun --nproc-per-node N -m paper_2512_09904_b300.serving sweep-sharded [--cases 64] [--steps 50]

Sweep: the paper's parametric study (shaft speed x immersion depth x oil
viscosity, Sec. 4) as 64 gear-bath cases of uneven size packed by case id in
one device array (sph_batch_*), every case advanced by the same CUDA-graph
launch per advection step.

Serve: a seeded Poisson stream of such requests.  Requests that arrive while
others run are admitted as soon as the batch has room (particle, cell and
case capacity = the HBM budget); finished cases hand back their torque and
heat-up curves and leave.  Both are compared with the plain per-case solver
(one sph_ctx after another, in arrival order) on the same inputs; each case's
result is checked to be identical in both.

Prints one JSON line.  Case geometry is generated before the clock starts
(it is the request payload); admission (host-to-device copy and sort),
stepping and curve read-back are timed.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from collections import deque

import numpy as np

from . import sph
from . import workloads as W


def _case(p):
    return W.gear_bath(dx=p["dx"], omega=p["omega"], depth_frac=p["depth_frac"], mu=p["mu"], seed=p["seed"])


def _sync():
    import torch
    torch.cuda.synchronize()


def _pct(x, q):
    return float(np.percentile(np.asarray(x), q)) if len(x) else float("nan")


def _result(b_or_ctx, slot=None, steps=0):
    if slot is None:
        th = b_or_ctx.sph_read_torque_heat(0)
        return th
    th = b_or_ctx.torque_heat(slot)
    th["curve"] = b_or_ctx.curve(slot, steps)
    return th


def batch_capacity(budget_bytes, max_cases, history_steps):
    """Largest particle capacity (sort cells = 6 x particles: a gear bath needs
    2.2-3.2 per particle) that fits the budget."""
    lo, hi = 1, 1 << 26
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if sph.Batch.bytes_for(mid, max_cases, 6 * mid + 1, history_steps) <= budget_bytes:
            lo = mid
        else:
            hi = mid - 1
    return lo, 6 * lo + 1


# ----------------------------------------------------------------- sweep ---
def sweep(n_cases=64, steps=50, count_scale=1.0, seed=4, sequential=True):
    reqs = W.sweep_cases(n_cases, seed=seed, count_scale=count_scale)
    cases = [_case(r) for r in reqs]
    n_fluid = np.array([c.n_fluid for c in cases])
    cap = int(sum(c.n_total for c in cases))
    cells = int(sum(sph.cells_of(c) for c in cases)) + 16
    out = dict(mode="sweep", cases=n_cases, steps=steps, count_scale=count_scale,
               n_fluid_total=int(n_fluid.sum()), n_particles_total=cap,
               n_fluid_range=[int(n_fluid.min()), int(n_fluid.max())])

    b = sph.Batch(cap, n_cases, cells, history_steps=steps)
    _sync()
    t0 = time.perf_counter()
    slots = [b.admit(c, steps) for c in cases]
    b.step(steps)
    res_b = [_result(b, s, steps) for s in slots]
    _sync()
    tb = time.perf_counter() - t0
    units = sum(int(c.n_fluid) * int(r["curve"][:, 6].sum()) for c, r in zip(cases, res_b))
    out["batched"] = dict(seconds=tb, cases_per_h=n_cases / tb * 3600.0, particle_substeps_per_s=units / tb,
                          kernels_per_step=b.info()["kernels_per_step"], hbm_bytes=b.bytes)
    b.close()
    if sequential:
        _sync()
        t0 = time.perf_counter()
        res_s = []
        for c in cases:
            ctx = sph.from_case(c)
            ctx.sph_step(steps)
            res_s.append(_result(ctx))
            ctx.close()
        _sync()
        ts = time.perf_counter() - t0
        out["sequential"] = dict(seconds=ts, cases_per_h=n_cases / ts * 3600.0, particle_substeps_per_s=units / ts)
        out["speedup_cases_per_h"] = out["batched"]["cases_per_h"] / out["sequential"]["cases_per_h"]
        out["max_abs_diff_torque_avg"] = max(abs(a["torque_avg"] - s["torque_avg"]) for a, s in zip(res_b, res_s))
        out["max_abs_diff_heat"] = max(abs(a["heat"] - s["heat"]) for a, s in zip(res_b, res_s))
    return out


def sweep_sharded(n_cases=64, steps=50, count_scale=1.0, seed=4):
    """The sweep over the ranks of one node (torchrun, one GPU per rank):
    whole cases assigned by particle count, each rank batches its share, the
    per-case torque / heat results are gathered on rank 0 (host objects)."""
    import os
    import torch
    import torch.distributed as dist
    from . import shard
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    reqs = W.sweep_cases(n_cases, seed=seed, count_scale=count_scale)
    cases = [_case(r) for r in reqs]
    owner = shard.assign_cases([c.n_total for c in cases], world)
    mine = [i for i in range(n_cases) if owner[i] == rank]
    local = {}
    t0 = time.perf_counter()
    if mine:
        cap = int(sum(cases[i].n_total for i in mine))
        cells = int(sum(sph.cells_of(cases[i]) for i in mine)) + 16
        b = sph.Batch(cap, len(mine), cells, history_steps=steps)
        slots = {i: b.admit(cases[i], steps) for i in mine}
        b.step(steps)
        for i, s in slots.items():
            th = b.torque_heat(s)
            local[i] = dict(torque_avg=th["torque_avg"], heat=th["heat"], mean_T=th["mean_T"])
        b.close()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    sec_max, _ = shard.reduce_timing(sec, 0.0, world, device="cuda")
    res = shard.gather_results(local, rank, world)
    if rank != 0:
        return None
    return dict(mode="sweep_sharded", ranks=world, cases=n_cases, steps=steps, seconds=sec_max,
                cases_per_h=n_cases / sec_max * 3600.0, results=[res[i] for i in range(n_cases)])


# ---------------------------------------------------------------- serving ---
def serve(n_requests=64, steps=200, rate=4.0, count_scale=1.0, seed=5, budget_gb=40.0, max_cases=16,
          steps_per_poll=8, sequential=True, policy="sjf"):
    """Serving loop over a seeded Poisson trace.  policy: "fifo" admits waiting
    requests in arrival order, "sjf" the one with the fewest particles first
    (a case never waits behind a larger one that arrived earlier)."""
    trace = W.serving_trace(n_requests, seed=seed, rate=rate, steps=steps, count_scale=count_scale)
    cases = [_case(r) for r in trace]
    arrivals = np.array([r["arrival"] for r in trace])
    n_fluid = np.array([c.n_fluid for c in cases])
    cap, cells = batch_capacity(budget_gb * 1e9, max_cases, steps)
    cap = max(cap, max(c.n_total for c in cases))
    out = dict(mode="serve", requests=n_requests, rate_per_s=rate, steps=steps, count_scale=count_scale,
               budget_gb=budget_gb, max_cases=max_cases, policy=policy,
               n_fluid_range=[int(n_fluid.min()), int(n_fluid.max())],
               n_fluid_mean=float(n_fluid.mean()))

    b = sph.Batch(cap, max_cases, cells, history_steps=steps)
    pending, resident = deque(), {}
    done_at = np.full(n_requests, np.nan)
    results = [None] * n_requests
    nxt, completed, max_resident, max_particles = 0, 0, 0, 0
    tm = dict(admit=0.0, step=0.0, poll=0.0, idle=0.0)
    _sync()
    t0 = time.perf_counter()
    while completed < n_requests:
        now = time.perf_counter() - t0
        while nxt < n_requests and arrivals[nxt] <= now:
            pending.append(nxt)
            nxt += 1
        ta = time.perf_counter()
        while pending:  # admission in policy order while the budget allows
            if policy == "sjf":
                k = min(range(len(pending)), key=lambda q: (cases[pending[q]].n_total, pending[q]))
                pending.rotate(-k)  # the chosen request to the front, the others keep their order
            r = pending[0]
            try:
                slot = b.admit(cases[r], steps)
            except sph.SphError as e:
                if policy == "sjf" and k:
                    pending.rotate(k)
                if e.status == sph.SPH_ENOMEM and resident:
                    break
                raise
            pending.popleft()
            if policy == "sjf" and k:
                pending.rotate(k)
            resident[slot] = r
        tb = time.perf_counter()
        tm["admit"] += tb - ta
        if not resident:
            time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
            tm["idle"] += time.perf_counter() - tb
            continue
        info = b.info()
        max_resident = max(max_resident, info["n_cases"])
        max_particles = max(max_particles, info["n_particles"])
        b.step(steps_per_poll)
        tc = time.perf_counter()
        tm["step"] += tc - tb
        for slot in list(resident):
            _, _, state = b.poll(slot)
            if state == sph.BATCH_RUNNING:
                continue
            r = resident.pop(slot)
            results[r] = _result(b, slot, steps)
            results[r]["state"] = state
            b.retire(slot)
            done_at[r] = time.perf_counter() - t0
            completed += 1
        tm["poll"] += time.perf_counter() - tc
    _sync()
    lat = done_at - arrivals
    span = float(np.nanmax(done_at) - arrivals[0])
    out["batched"] = dict(cases_per_h=n_requests / span * 3600.0, p50_latency_s=_pct(lat, 50),
                          p99_latency_s=_pct(lat, 99), makespan_s=span, max_resident_cases=max_resident,
                          max_resident_particles=max_particles, hbm_bytes=b.bytes,
                          unstable=int(sum(1 for r in results if r["state"] == sph.BATCH_UNSTABLE)),
                          loop_seconds={k: round(v, 3) for k, v in tm.items()})
    b.close()
    if sequential:
        # the plain per-case solver on the same trace: one case at a time
        done_s = np.full(n_requests, np.nan)
        res_s = []
        _sync()
        t0 = time.perf_counter()
        tms = dict(create=0.0, step=0.0, idle=0.0)
        for r in range(n_requests):
            now = time.perf_counter() - t0
            if now < arrivals[r]:
                time.sleep(arrivals[r] - now)
                tms["idle"] += arrivals[r] - now
            tc0 = time.perf_counter()
            ctx = sph.from_case(cases[r])
            tms["create"] += time.perf_counter() - tc0
            state = sph.BATCH_DONE
            done = 0
            while done < steps:  # same poll granularity as the batch: stop at an instability
                k = min(steps_per_poll, steps - done)
                try:
                    ctx.sph_step(k)
                except sph.SphError as e:
                    if e.status != sph.SPH_EUNSTABLE:
                        raise
                    state = sph.BATCH_UNSTABLE
                    break
                done += k
            res = _result(ctx)
            res["state"] = state
            res_s.append(res)
            ctx.close()
            done_s[r] = time.perf_counter() - t0
        lat_s = done_s - arrivals
        span_s = float(np.nanmax(done_s) - arrivals[0])
        out["sequential"] = dict(cases_per_h=n_requests / span_s * 3600.0, p50_latency_s=_pct(lat_s, 50),
                                 p99_latency_s=_pct(lat_s, 99), makespan_s=span_s,
                                 loop_seconds={k: round(v, 3) for k, v in tms.items()})
        out["speedup_cases_per_h"] = out["batched"]["cases_per_h"] / out["sequential"]["cases_per_h"]
        ok = [(a, s) for a, s in zip(results, res_s) if a["state"] != sph.BATCH_UNSTABLE]
        out["sequential"]["unstable"] = int(sum(1 for s in res_s if s["state"] == sph.BATCH_UNSTABLE))
        out["state_mismatches"] = int(sum(1 for a, s in zip(results, res_s) if a["state"] != s["state"]))
        out["max_abs_diff_torque_avg"] = max((abs(a["torque_avg"] - s["torque_avg"]) for a, s in ok), default=None)
        out["max_abs_diff_heat"] = max((abs(a["heat"] - s["heat"]) for a, s in ok), default=None)
    out["unstable_requests"] = [dict(i=i, **{k: trace[i][k] for k in ("omega", "depth_frac", "mu", "n_fluid", "dx")})
                                for i, r in enumerate(results) if r["state"] == sph.BATCH_UNSTABLE]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["sweep", "serve", "sweep-sharded"])
    ap.add_argument("--cases", type=int, default=64)
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--rate", type=float, default=4.0)
    ap.add_argument("--count-scale", type=float, default=0.0)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--no-sequential", action="store_true")
    ap.add_argument("--max-cases", type=int, default=16, help="resident cases at most (serve)")
    ap.add_argument("--policy", default="sjf", choices=["fifo", "sjf"], help="admission order (serve)")
    a = ap.parse_args(argv)
    import os
    import torch
    if a.mode == "sweep-sharded":
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        if int(os.environ.get("WORLD_SIZE", "1")) > 1:
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        r = sweep_sharded(a.cases, a.steps or 50, a.count_scale or 1.0)
        if r is not None:
            print(json.dumps(r), flush=True)
        if dist.is_initialized():
            dist.destroy_process_group()
        return
    torch.cuda.set_device(0)
    if a.mode == "sweep":
        r = sweep(a.cases, a.steps or 50, a.count_scale or 1.0, sequential=not a.no_sequential)
    else:
        r = serve(a.requests, a.steps or 200, a.rate, a.count_scale or 1.0, budget_gb=a.budget_gb,
                  max_cases=a.max_cases, sequential=not a.no_sequential, policy=a.policy)
    print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
