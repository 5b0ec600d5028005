"""A bounded solver run for profilers: one mesh, one state, a few time steps.

    python -m paper_2204_03575_gb300.profile_case --nx 1024 --ny 1024 --steps 1 --restart 10
    python -m paper_2204_03575_gb300.profile_case --batch 64 --precision 1 --restart 30 --warmup 0 --steps 2
    python -m paper_2204_03575_gb300.profile_case --nx 128 --ny 128 --nz 32 --potential 3 --steps 1
    python -m paper_2204_03575_gb300.profile_case --nx 512 --ny 512 --steps 1 --project 1024
    python -m paper_2204_03575_gb300.profile_case --nx 256 --ny 256 --steps 3 --ws 4

Builds the mesh, system, preconditioner and state on cuda:0 (seeded initial state, paper
parameters), runs the warm-up and timed steps and prints per-step statistics; with --project G,
then projects the final 2D morphology onto a G x G grid (Section 5); with --ws B, runs the
warm-start network (seeded random weights) on the last three states: one prediction and one
training step on a batch of B copies.  Used as the
target of ncu captures, where the full benchmark would hold too much device memory.
"""
import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--nz", type=int, default=0)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--restart", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--potential", type=int, default=0)
    ap.add_argument("--graphs", type=int, default=1,
                    help="0: host-driven Krylov loop with direct launches (ncu profiles no kernel inside a "
                         "graph that holds conditional nodes)")
    ap.add_argument("--precond-m", type=int, default=0)
    ap.add_argument("--pdl", type=int, default=1, help="0: plain stream-ordered launches")
    ap.add_argument("--ws", type=int, default=0, help="batch of a warm-start network prediction and training step")
    ap.add_argument("--ws-engine", type=int, default=1, help="warm-start convolutions: 0 mma.sync, 1 tcgen05")
    ap.add_argument("--project", type=int, default=0, help="grid size of a final morphology projection")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead of one mesh: this many runs of inputs.batch_runs(n, seed=0)")
    a = ap.parse_args()
    import torch
    from paper_2204_03575_gb300 import ch
    torch.cuda.set_device(0)
    kw = dict(nx=a.nx, ny=a.ny, precision=a.precision, restart=a.restart, potential=a.potential,
              precond_M=a.precond_m, graphs=a.graphs, pdl=a.pdl)
    if a.nz:
        kw.update(dim=3, nz=a.nz, Lz=a.nz / a.nx)
    if a.batch:
        from paper_2204_03575_gb300 import inputs
        spec = inputs.batch_runs(a.batch, seed=0)
        p = ch.Params(precision=a.precision, restart=a.restart, graphs=a.graphs, pdl=a.pdl)
        mesh = ch.Mesh(p, runs=[ch.Params(nx=nx, ny=ny) for nx, ny, _, _ in spec])
        system = ch.System(mesh, p)
        pc = ch.Precond(system)
        state = ch.State(system, pc)
        state.init_seeded_batch([x[2] for x in spec], [x[3] for x in spec], 0.01, seed=0)
    else:
        p = ch.Params(**kw)
        system = ch.System(ch.Mesh(p), p)
        pc = ch.Precond(system)
        state = ch.State(system, pc)
        state.init_seeded(0.33, 0.33, 0.01, seed=0)
    for _ in range(a.warmup):
        state.step()
    hist = []
    ms, its = [], []
    for k in range(a.steps):
        s = state.step()
        ms.append(s["ms"])
        its.append(sum(s["iters"]))
        print(json.dumps({"step": k, **s}), flush=True)
        if a.ws and not a.batch and not a.nz:
            g = state.get()
            hist = (hist + [torch.stack([g["phi_p"], g["phi_nfa"], g["mu_p"], g["mu_nfa"]], 1).contiguous()])[-3:]
    if a.steps:
        print(json.dumps({"steps": a.steps, "mean_ms": sum(ms) / len(ms), "iters": sum(its)}), flush=True)
    if a.ws and len(hist) == 3:
        import numpy as np
        net = ch.WarmStartNet(a.ny + 1, a.nx + 1, max_batch=a.ws)
        net.set_engine(a.ws_engine)
        net.set_params((np.random.default_rng(0).standard_normal(ch.lib().ch_ws_nparams()) * 0.1).astype(np.float32))
        q2, q, s4 = hist
        pred = net.predict(s4, q, q2)
        batch = [t.float().unsqueeze(0).repeat(a.ws, 1, 1).contiguous() for t in (s4, q, q2, 2 * s4 - q)]
        loss = net.train_step(*batch, 0.0)
        torch.cuda.synchronize()
        print(json.dumps({"ws_batch": a.ws, "pred_finite": bool(torch.isfinite(pred).all()), "loss": loss}),
              flush=True)
    if a.project and not a.batch and not a.nz:
        g = state.get()
        polymer, _, _ = ch.morphology_project(g["phi_p"], g["phi_nfa"], a.nx, a.ny, 1.0, 1.0, a.project, a.project)
        torch.cuda.synchronize()
        print(json.dumps({"project": a.project, "polymer_fraction": float(polymer.float().mean())}), flush=True)


if __name__ == "__main__":
    main()
