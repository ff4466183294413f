"""GPU-side helpers for the tests: pack seeded problems, call the C ABI through the binding, return numpy."""
from __future__ import annotations

import numpy as np


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def eigh_batch(ctx, problems, a_words):
    import paper_2402_11868_gb300 as Z
    torch, dev = torch_dev()
    ns = [p.n for p in problems]
    a_off, w_off, tot_a, tot_w = Z.batch_offsets(ns)
    A = torch.from_numpy(Z.pack([p.A for p in problems], a_words)).to(dev)
    W = torch.zeros(tot_w, dtype=torch.float64, device=dev)
    V = torch.zeros(tot_a * 2, dtype=torch.float64, device=dev)
    info = torch.full((len(ns),), -7, dtype=torch.int32, device=dev)
    Z.zkq_eigh_batched(ctx, ns, a_off, A, a_words, W, V, info)
    torch.cuda.synchronize()
    return dict(A=A, W=W, V=V, info=info, ns=ns, a_off=a_off, w_off=w_off)


def refine_batch(ctx, problems, a_words, target, method, eig=None):
    import paper_2402_11868_gb300 as Z
    torch, dev = torch_dev()
    if eig is None:
        eig = eigh_batch(ctx, problems, a_words)
    ns, a_off, w_off = eig["ns"], eig["a_off"], eig["w_off"]
    tot_w = sum(ns); tot_a = sum(n * n for n in ns)
    Wo = torch.zeros(tot_w * target, dtype=torch.float64, device=dev)
    Vo = torch.zeros(tot_a * 2 * target, dtype=torch.float64, device=dev)
    err = torch.zeros(tot_w, dtype=torch.float64, device=dev)
    info = torch.full((len(ns),), -7, dtype=torch.int32, device=dev)
    Z.zkq_rqi_refine(ctx, ns, a_off, eig["A"], a_words, eig["W"], eig["V"], target, method, Wo, Vo, err, info)
    torch.cuda.synchronize()
    out = dict(eig)
    out.update(Wo=Wo, Vo=Vo, err=err, rinfo=info, target=target)
    return out


def problem_views(res, b, words=None):
    """(lam words (n, w), V words (n*n, 2, w)) of problem b from a refine or eigh result, as numpy."""
    n = res["ns"][b]
    if words is None:       # FP64 stage
        W = res["W"].cpu().numpy()[res["w_off"][b]:res["w_off"][b] + n].reshape(n, 1)
        V = res["V"].cpu().numpy()[2 * res["a_off"][b]:2 * (res["a_off"][b] + n * n)].reshape(n * n, 2, 1)
        return W, V
    t = words
    W = res["Wo"].cpu().numpy()[t * res["w_off"][b]:t * (res["w_off"][b] + n)].reshape(n, t)
    V = res["Vo"].cpu().numpy()[2 * t * res["a_off"][b]:2 * t * (res["a_off"][b] + n * n)].reshape(n * n, 2, t)
    return W, V
