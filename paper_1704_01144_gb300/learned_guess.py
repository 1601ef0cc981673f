"""Training pipeline of the learned starting guess of the exact Riemann
solver (harvest -> label -> train -> held-out evaluation).

Every step runs in the library's CUDA kernels through its C ABI:
``fv_harvest_pairs`` takes Riemann pairs from a mesh's own reconstructed face
states between cycles of its run, ``fv_mlp_label`` solves them exactly in
FP64 and forms features and targets, ``fv_mlp_train`` trains the network with
the FP32 forward/backward/Adam kernels, and the evaluation runs the flux
kernel with either guess.  numpy only draws the held-out split and lists the
samples past the gate.
"""
from __future__ import annotations

import numpy as np

from . import fv

DEFAULT_GATE = 0.02


def harvest(mesh: "fv.Mesh", prim, cycles: int, per_cycle: int, seed: int, stream=None):
    """Run `cycles` cycles of the mesh from `prim`, harvesting `per_cycle`
    pairs after each; returns a (cycles*per_cycle, 6) float64 CUDA tensor."""
    import torch
    mesh.set_state(prim)
    per_cycle = min(int(per_cycle), mesh.nf)
    out = torch.empty((cycles * per_cycle, 6), dtype=torch.float64, device="cuda")
    for c in range(cycles):
        mesh.advance(1, stream=stream, want_time=False)
        fv.fv_harvest_pairs(mesh.h, per_cycle, seed * 100003 + c, out=out[c * per_cycle:(c + 1) * per_cycle],
                            stream=stream)
    torch.cuda.synchronize()
    st = mesh.status()
    if st != 0:
        raise RuntimeError(f"harvest run failed: {fv.fv_last_error()}")
    return out


def face_frame(pairs):
    """Face-frame pairs (n, 6) -> (WL, WR, normals) for the flux batch entry
    points: normal (1, 0, 0), tangential velocity 0."""
    import torch
    n = pairs.shape[0]
    WL = torch.zeros((5, n), dtype=torch.float64, device=pairs.device)
    WR = torch.zeros_like(WL)
    WL[0], WL[1], WL[4] = pairs[:, 0], pairs[:, 1], pairs[:, 2]
    WR[0], WR[1], WR[4] = pairs[:, 3], pairs[:, 4], pairs[:, 5]
    nrm = torch.zeros((3, n), dtype=torch.float64, device=pairs.device)
    nrm[0] = 1.0
    return WL, WR, nrm


def train(pairs, target=fv.FV_MLP_TARGET_TR, gate=DEFAULT_GATE, holdout=0.1, epochs=20, batch=4096,
          lr0=3e-3, lr1=3e-5, seed=1):
    """Label the pairs, split off a held-out tenth, train on the training
    pairs past the gate.  Returns (params float32 CUDA tensor, info dict)."""
    import torch
    x, y, ps, q = fv.fv_mlp_label(pairs, target, want_q=True)
    n = pairs.shape[0]
    perm = np.random.default_rng(seed).permutation(n)
    n_te = int(n * holdout)
    te, tr = perm[:n_te], perm[n_te:]
    qh = q.cpu().numpy()
    sel = tr[qh[tr] > gate] if gate >= 0 else tr
    if len(sel) == 0:
        raise RuntimeError("no training pair past the gate")
    params = torch.from_numpy(fv.fv_mlp_init(seed)).cuda()
    hist = fv.fv_mlp_train(params, x, y, sel=sel, epochs=epochs, batch=batch, lr0=lr0, lr1=lr1,
                           seed=seed)
    info = {"pairs": int(n), "train_pairs_past_gate": int(len(sel)), "heldout_pairs": int(n_te),
            "gate": gate, "target": int(target), "epochs": epochs, "batch": batch,
            "steps": int(len(hist)), "loss_first": float(hist[0]), "loss_last": float(hist[-1])}
    return params, {"info": info, "x": x, "y": y, "q": qh, "heldout": te, "train": sel}


def evaluate(params, pairs, data, target=fv.FV_MLP_TARGET_TR, gate=DEFAULT_GATE, precision=fv.FV_FP64):
    """Held-out comparison of the two guesses: mean |log(p_guess/p*)| where
    the gate passes, and mean Newton iterations to the same tolerance there
    and over all held-out pairs."""
    import torch
    te = data["heldout"]
    q = data["q"]
    gated = te[q[te] > gate] if gate >= 0 else te
    pk = fv.fv_mlp_pack(params, target, gate=gate)
    cfg = fv.fv_config_default(precision=precision)
    res = {"heldout_pairs": int(len(te)), "past_gate": int(len(gated)), "precision":
           "fp64" if precision == fv.FV_FP64 else "fp32"}
    for name, idx in (("past_gate", gated), ("all", te)):
        if len(idx) == 0:
            continue
        it = torch.from_numpy(idx).cuda()
        WL, WR, nrm = face_frame(pairs[it])
        _, i_tr = fv.fv_godunov_flux_batch(WL, WR, nrm, cfg)
        _, i_ml = fv.fv_godunov_flux_batch_mlp(WL, WR, nrm, cfg, pk)
        if bool((i_tr < 0).any()) or bool((i_ml < 0).any()):
            raise RuntimeError("Riemann solver failed on held-out pairs")
        res[f"newton_iters_{name}"] = {"two_rarefaction": round(i_tr.double().mean().item(), 4),
                                       "learned": round(i_ml.double().mean().item(), 4)}
    if len(gated) and target == fv.FV_MLP_TARGET_TR:
        g = torch.from_numpy(gated).cuda()
        y = data["y"][g].double()
        pred = fv.fv_mlp_infer(pk, data["x"][g].contiguous()).double()
        qg = torch.from_numpy(q[gated]).cuda().double()
        sc = (qg / (1 + qg)) ** 3
        res["guess_log_err_past_gate"] = {"two_rarefaction": (sc * y).abs().mean().item(),
                                          "learned": (sc * (pred - y)).abs().mean().item()}
    return res
