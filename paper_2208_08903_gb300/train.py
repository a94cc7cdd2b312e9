"""Reverse-KL self-training driver (the paper's Sec. 3 training loop).

for epoch in epochs: for it in iterations: draw a batch from the prior, take
the gradient of the shifted reverse KL loss, apply Adam -- each iteration is
one gf_flow_train_step call (forward with saved layer inputs, hand-written
backward, Adam on the device).  Prior counters advance with every iteration,
so a run is reproducible from (seed, epochs, iterations, batch).
"""
from __future__ import annotations

import dataclasses

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
          betas=(0.9, 0.999), eps: float = 1e-8) -> TrainState:
    """Runs epochs x iterations Adam steps of the reverse-KL loss; returns the
    state (step count, Adam moments, recorded losses) so training can resume."""
    st = state or new_state(flow)
    dev = st.adam_m.device
    ws = torch.empty(max(flow.train_workspace_bytes(batch), 1), device=dev, dtype=torch.uint8)
    pending = []
    for _ in range(epochs):
        for _ in range(iterations):
            st.step += 1
            loss, _ = flow.train_step(batch, phi4, seed=seed, counter0=st.step * batch, lr=lr,
                                      adam_m=st.adam_m, adam_v=st.adam_v, adam_t=st.step,
                                      beta1=betas[0], beta2=betas[1], adam_eps=eps, grad=False,
                                      workspace=ws)
            if st.step % record_every == 0:
                pending.append(loss)
    if pending:
        st.losses.extend(torch.cat(pending).cpu().tolist())
    return st
