"""Reverse-KL self-training driver (the paper's Sec. 3 training loop).

for epoch in epochs: for it in iterations: draw a batch from the prior, take
the gradient of the shifted reverse KL loss, apply Adam -- each iteration is
one gf_flow_train_step call (forward with saved layer inputs, hand-written
backward, Adam on the device).  Prior counters advance with every iteration,
so a run is reproducible from (seed, epochs, iterations, batch), and a run
resumed from a checkpoint continues bit for bit where it stopped.

The paper's training settings (Sec. 3, the example configuration) map to:
seed -> `seed`, batchsize -> `batch`, epochs / iterations, base_lr -> `lr`,
opt = Adam, lr_scheduler -> `lr_schedule` (a function of the 1-based step;
None = constant), pretrained -> `load_checkpoint` + `state=`.

Command line (trains, checkpoints, evaluates acceptance and ESS per epoch):
    python -m paper_2208_08903_gb300.train --workload c1 --epochs 200 --iterations 100
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time

import numpy as np
import torch

from . import api


@dataclasses.dataclass
class TrainState:
    step: int
    adam_m: torch.Tensor
    adam_v: torch.Tensor
    losses: list


def new_state(flow: api.Flow) -> TrainState:
    dev = torch.device("cuda", torch.cuda.current_device())
    return TrainState(0, torch.zeros(flow.n_params, device=dev), torch.zeros(flow.n_params, device=dev), [])


def train(flow: api.Flow, phi4, epochs: int, iterations: int, batch: int, lr: float = 1e-3,
          seed: int = 12345, state: TrainState | None = None, record_every: int = 1,
          betas=(0.9, 0.999), eps: float = 1e-8, lr_schedule=None) -> TrainState:
    """Runs epochs x iterations Adam steps of the reverse-KL loss; returns the
    state (step count, Adam moments, recorded losses) so training can resume.
    lr_schedule(step) -> learning rate overrides `lr` when given."""
    st = state or new_state(flow)
    dev = st.adam_m.device
    ws = torch.empty(max(flow.train_workspace_bytes(batch), 1), device=dev, dtype=torch.uint8)
    pending = []
    for _ in range(epochs):
        for _ in range(iterations):
            st.step += 1
            step_lr = lr if lr_schedule is None else float(lr_schedule(st.step))
            loss, _ = flow.train_step(batch, phi4, seed=seed, counter0=st.step * batch, lr=step_lr,
                                      adam_m=st.adam_m, adam_v=st.adam_v, adam_t=st.step,
                                      beta1=betas[0], beta2=betas[1], adam_eps=eps, grad=False,
                                      workspace=ws)
            if st.step % record_every == 0:
                pending.append(loss)
    if pending:
        st.losses.extend(torch.cat(pending).cpu().tolist())
    return st


def save_checkpoint(path: str, flow: api.Flow, state: TrainState, **meta) -> None:
    """Writes the flow's FP32 weights, the Adam moments, the step count, the
    recorded losses, the flow shape and any extra metadata to an .npz file."""
    sh = flow.shape
    np.savez(path,
             weights=flow.get_weights().cpu().numpy(),
             adam_m=state.adam_m.cpu().numpy(), adam_v=state.adam_v.cpu().numpy(),
             step=np.int64(state.step), losses=np.asarray(state.losses, dtype=np.float64),
             shape=np.array([sh.nd, sh.L, sh.n_layers, sh.c1, sh.c2, int(bool(sh.use_final_tanh))],
                            dtype=np.int64),
             leaky_slope=np.float64(sh.leaky_slope),
             meta=json.dumps(meta))


def load_checkpoint(path: str, flow: api.Flow) -> tuple[TrainState, dict]:
    """Loads a checkpoint into `flow` (shapes must match) and returns the
    training state to pass to `train(state=...)` and the stored metadata."""
    z = np.load(path)
    sh = flow.shape
    want = [sh.nd, sh.L, sh.n_layers, sh.c1, sh.c2, int(bool(sh.use_final_tanh))]
    if z["shape"].tolist() != want or float(z["leaky_slope"]) != float(sh.leaky_slope):
        raise ValueError(f"checkpoint shape {z['shape'].tolist()} does not match the flow {want}")
    dev = torch.device("cuda", torch.cuda.current_device())
    flow.set_weights(torch.tensor(z["weights"], dtype=torch.float32, device=dev))
    st = TrainState(int(z["step"]), torch.tensor(z["adam_m"], device=dev), torch.tensor(z["adam_v"], device=dev),
                    z["losses"].tolist())
    return st, json.loads(str(z["meta"]))


CHECKPOINT_DIR = __import__("os").path.join(__import__("os").path.dirname(__file__), "checkpoints")


def load_weights(path: str, shape=None):
    """FP64 canonical weights of a weights-only checkpoint (the `weights`,
    `shape`, `leaky_slope` entries of an .npz written by save_checkpoint or
    shipped in checkpoints/); checks the stored shape against `shape`."""
    z = np.load(path)
    if shape is not None:
        want = [shape.nd, shape.L, shape.n_layers, shape.c1, shape.c2, int(bool(shape.use_final_tanh))]
        if z["shape"].tolist() != want or float(z["leaky_slope"]) != float(shape.leaky_slope):
            raise ValueError(f"checkpoint shape {z['shape'].tolist()} does not match {want}")
    return z["weights"].astype(np.float64)


def evaluate(flow: api.Flow, phi4, n_proposals: int, batch: int, seed: int, counter0: int = 0,
             mh_seed: int = 1, sampler: str = "fused", keep_logw: bool = False) -> dict:
    """Acceptance of an MH independence chain over n_proposals flow samples,
    the ESS fraction of their importance weights and the chain average of
    |M| with its integrated autocorrelation time (all on the device).
    sampler: "fused" (gf_flow_sample of `flow`, whatever its precision) or
    "unfused" (one kernel per conv).  The proposals are fixed by (seed,
    counter0): two flows evaluated with the same arguments see the same prior
    samples and the same MH uniforms."""
    st = api.new_mh_state(mh_seed)
    lws, Ms, idxs = [], [], []
    ws = None
    t0 = time.perf_counter()
    for i in range(0, n_proposals, batch):
        b = min(batch, n_proposals - i)
        if sampler == "fused":
            r = flow.sample(b, seed=seed, counter0=counter0 + i, phi4=phi4)
        else:
            if ws is None:
                ws = torch.empty(flow.unfused_workspace_bytes(batch), device="cuda", dtype=torch.uint8)
            r = flow.sample_unfused(b, seed=seed, counter0=counter0 + i, phi4=phi4, workspace=ws)
        idx, _ = api.mh_chain(st, r.logw)
        M, _ = api.observables(flow.shape.nd, flow.shape.L, r.phi, two_point=False)
        lws.append(r.logw)
        Ms.append(M)
        idxs.append(idx)
    logw = torch.cat(lws)
    series = api.chain_gather(torch.cat(idxs), torch.cat(Ms)).abs().contiguous()
    t_max = int(min(1000, max(0, n_proposals - 1)))
    _, summ = api.autocorr(series, t_max)
    ess = api.ess(logw)
    s = api.read_mh_state(st)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    summ = summ.cpu().tolist()
    n = max(1, s.step - 1)
    acc = s.n_acc / n
    out = {"acceptance": acc, "acceptance_binomial_err": math.sqrt(max(acc * (1 - acc), 0.0) / n),
           "ess": float(ess.item()), "abs_M": summ[3], "tau_int_abs_M": summ[0],
           "tau_int_err": summ[2], "window": int(summ[1]), "proposals": n_proposals,
           "seconds": secs, "precision": getattr(flow, "precision", "fp32"), "sampler": sampler}
    if keep_logw:
        out["logw"] = logw
        out["chain_idx"] = torch.cat(idxs)
    return out


def decision_agreement(a: dict, b: dict) -> float:
    """Fraction of proposals on which two evaluations (kept with keep_logw)
    left their chains in the same state."""
    return float((a["chain_idx"] == b["chain_idx"]).double().mean().item())


def main(argv=None):
    import gf_inputs as gi
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="c1", choices=["c1", "c2", "c3"])
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--iterations", type=int, default=100)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=12345)
    ap.add_argument("--model-seed", type=int, default=2021)
    ap.add_argument("--checkpoint", default="")
    ap.add_argument("--resume", default="")
    ap.add_argument("--eval-proposals", type=int, default=16384)
    ap.add_argument("--eval-every", type=int, default=20)
    ap.add_argument("--n-layers", type=int, default=0, help="override the workload's coupling-layer count")
    ap.add_argument("--m2", type=float, default=None)
    ap.add_argument("--lam", type=float, default=None)
    ap.add_argument("--compare-proposals", type=int, default=0,
                    help="proposals for the final sampler comparison (default: --eval-proposals)")
    args = ap.parse_args(argv)
    W = gi.WORKLOADS[args.workload]
    shape, phi4 = W["shape"], W["phi4"]
    if args.n_layers:
        shape = dataclasses.replace(shape, n_layers=args.n_layers)
    if args.m2 is not None or args.lam is not None:
        phi4 = gi.Phi4(args.m2 if args.m2 is not None else phi4.m2, args.lam if args.lam is not None else phi4.lam)
    batch = args.batch or (64 if args.workload == "c3" else W["batch"])
    flow = api.Flow(shape, gi.init_weights(shape, seed=args.model_seed))
    state = None
    if args.resume:
        state, _ = load_checkpoint(args.resume, flow)
    t0 = time.perf_counter()
    for ep in range(args.epochs):
        state = train(flow, phi4, 1, args.iterations, batch, lr=args.lr, seed=args.seed, state=state)
        if (ep + 1) % args.eval_every == 0 or ep + 1 == args.epochs:
            ev = evaluate(flow, phi4, args.eval_proposals, 4096, seed=args.seed + 1, counter0=state.step << 20)
            line = {"epoch": ep + 1, "step": state.step, "loss": float(np.mean(state.losses[-args.iterations:])),
                    "seconds": time.perf_counter() - t0, **ev}
            print(json.dumps(line), flush=True)
            if args.checkpoint:
                save_checkpoint(args.checkpoint, flow, state, workload=args.workload, seed=args.seed,
                                batch=batch, lr=args.lr)
    # the fused and the plain (one kernel per convolution) FP32 samplers, and the
    # BF16 tensor-core sampler where the shape has one, on the same proposals
    n_cmp = args.compare_proposals or args.eval_proposals
    arms = {"fused": (flow, "fused"), "unfused": (flow, "unfused")}
    if (shape.nd, shape.L, shape.c1, shape.c2) == (3, 16, 32, 32) and shape.is_default_net:
        wt = flow.get_weights().double().cpu().numpy()
        arms["bf16"] = (api.Flow(shape, wt, precision="bf16"), "fused")
    same = {k: evaluate(f, phi4, n_cmp, 4096, seed=args.seed + 2, sampler=kind, keep_logw=True)
            for k, (f, kind) in arms.items()}
    line = {"final": True, "step": state.step, "theory": [phi4.m2, phi4.lam], "n_layers": shape.n_layers}
    for k, ev in same.items():
        line[k] = {kk: v for kk, v in ev.items() if kk not in ("logw", "chain_idx")}
        line[k]["configs_per_s"] = n_cmp / ev["seconds"]
        if k != "fused":
            line[k]["decisions_same_as_fused"] = decision_agreement(ev, same["fused"])
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
