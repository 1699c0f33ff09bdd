"""Training of the learned correction of the circulant preconditioner.

The correction is a U-Net U applied after M_C inside flexible CG:
z = M_C r, z <- z + ||z|| U(z / ||z||).  It is trained on pairs harvested from
converged FP64 solves: at iterate k of PCG with M_C, the residual r_k and the
error e_k = x* - x_k satisfy A e_k = r_k, so the ideal preconditioner output is
e_k; with z_k = M_C r_k and s_k = ||z_k|| the network input is z_k / s_k and its
target (e_k - z_k) / s_k.

Every numerical step (solves, preconditioner applications, network forward,
backward and Adam) runs in the library's CUDA kernels through ``cmm``; this
module only orders the calls and batches the data.
"""
from __future__ import annotations

import torch

from . import cmm


def harvest_pairs(op, pc, b, max_iter=200, tol=1e-10, every=1, solve_pc=None, window=1):
    """Runs FP64 PCG with the (circulant) preconditioner pc on A x = b and returns
    (inputs, targets, info): FP32 tensors [K, 3, ny, nx] of normalised pairs from the
    snapshots k = 0, every, ... of the solve.  With solve_pc (e.g. M_C followed by
    the current network) the iterates come from that flexible solve instead (FCG(m)
    with window m > 1), while the pairs are still formed with z = M_C r, so a network
    can be retrained on the residuals it meets itself."""
    slots = max_iter // every + 1
    snaps = torch.zeros((slots, 2) + tuple(op.shape), dtype=torch.float64, device=b.device)
    x = op.new_map()
    run_pc = solve_pc if solve_pc is not None else pc
    info = cmm.cmm_solve(op.h, run_pc.h, b, x, tol, 20 * max_iter + 200, 10, True, False, None, None,
                         snapshots=snaps, snapshot_every=every, flexible=window > 1, window=window)
    taken = min(slots, info.iterations // every + 1)
    ins = torch.empty((taken,) + tuple(op.shape), dtype=torch.float32, device=b.device)
    tgts = torch.empty_like(ins)
    cmm.cmm_harvest_pairs(pc.h, snaps, taken, x, ins, tgts)
    return ins, tgts, info


def train(net: "cmm.UNet", inputs, targets, epochs=5, batch=32, lr=1e-3, seed=0, val=None, log=None):
    """Adam on the pairs; returns the list of (epoch, mean train loss, val loss)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = inputs.shape[0]
    hist = []
    for ep in range(epochs):
        order = torch.randperm(n, generator=g).to(inputs.device)
        tot, cnt = 0.0, 0
        for i0 in range(0, n - batch + 1, batch):
            idx = order[i0:i0 + batch]
            xb = inputs.index_select(0, idx).contiguous()
            tb = targets.index_select(0, idx).contiguous()
            tot += cmm.cmm_unet_train_step(net.h, xb, tb, lr)
            cnt += 1
        vl = None
        if val is not None:
            vi, vt = val
            vls = [cmm.cmm_unet_loss_grad(net.h, vi[j:j + batch].contiguous(), vt[j:j + batch].contiguous())
                   for j in range(0, vi.shape[0] - batch + 1, batch)]
            vl = sum(vls) / max(1, len(vls))
        hist.append((ep, tot / max(1, cnt), vl))
        if log:
            log(f"epoch {ep}: train {tot / max(1, cnt):.4e} val {vl}")
    return hist
