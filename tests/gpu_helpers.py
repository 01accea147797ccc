"""Shared helpers of the GPU tests: build a plan and the matching oracle plan from one problem."""
import numpy as np
import torch

import oracle as O
import synth


def mm():
    import paper_2112_03370_gb300.mm as m
    return m


def plans(prob: synth.Problem, precision=0, algo=0, cond_max=1e3, on_device=True, tile_steps=0, pt_sub=0):
    m = mm()
    dev = torch.device("cuda")
    if on_device:
        pix, psi, band = prob.pix.to(dev), prob.psi.to(dev), prob.band.to(dev)
    else:
        pix, psi, band = prob.pix.cpu(), prob.psi.cpu(), prob.band.cpu()
    gp = m.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, pix.contiguous(),
                   psi.contiguous(), prob.lam, band.contiguous(), cond_max=cond_max,
                   precision=precision, toeplitz_algo=algo, tile_steps=tile_steps, pt_sub=pt_sub)
    nb = synth.to_numpy(prob)
    op = O.make_plan(nb["pix"], nb["psi"], nb["block_len"], nb["band"], nb["n_pix"],
                     cond_max=cond_max)
    return gp, op, nb


def rel_max(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
