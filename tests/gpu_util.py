"""Helpers for GPU tests: move seeded channels to the device in the C-ABI
layout, run the library, bring the results back as complex128 matrices."""
from __future__ import annotations

import numpy as np

from paper_2305_13925_gb300 import binding


def rel_fro(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_F / ||b||_F, the parity metric for W."""
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(H: np.ndarray, torch, pad_even: bool = True):
    """(M, K) complex -> device complex64 tensor of shape (K, ld) with ld even."""
    M, K = H.shape
    ld = M + (M & 1) if pad_even else M
    t = torch.zeros((K, ld), dtype=torch.complex64)
    t[:, :M] = torch.from_numpy(np.ascontiguousarray(H.T).astype(np.complex64))
    return t.cuda()[:, :M]


def to_dev_bf16(H: np.ndarray, torch):
    """(M, K) complex with bfloat16-exact parts -> device bfloat16 (K, ld, 2), ld % 4 == 0."""
    M, K = H.shape
    ld = (M + 3) // 4 * 4
    t = torch.zeros((K, ld, 2), dtype=torch.float32)
    t[:, :M, 0] = torch.from_numpy(np.ascontiguousarray(H.T.real).astype(np.float32))
    t[:, :M, 1] = torch.from_numpy(np.ascontiguousarray(H.T.imag).astype(np.float32))
    return t.to(torch.bfloat16).cuda()[:, :M, :]


def run(Hs, xis, variant="standard", T=6, tol=0.0, want_X=False, want_A=False, power=1.0,
        plan=False, graph=False, repeats=1, precision="fp32", prec=None, bf16=False,
        refine_sweeps=0, want_hist=False, refine_fp64=False, simt_iteration=False, refine_tol=0.0,
        refine_solve_tol=0.0, omegas=None, refine_selective=False, refine_residual=None):
    """Precode each (M_i, K_i) channel of ``Hs`` in one batch on the GPU."""
    import torch
    n = len(Hs)
    Hd = [to_dev_bf16(h, torch) if bf16 else to_dev(h, torch) for h in Hs]
    Wd = [to_dev(np.full(h.shape, np.nan, dtype=np.complex128), torch) for h in Hs]
    Xd = [torch.zeros((h.shape[1], h.shape[1]), dtype=torch.complex64, device="cuda") for h in Hs] if want_X else None
    Ad = [torch.zeros((h.shape[1], h.shape[1]), dtype=torch.complex64, device="cuda") for h in Hs] if want_A else None
    hist = [torch.full((refine_sweeps + 1,), -1.0, device="cuda") for _ in Hs] if want_hist else None
    insts = [binding.instance(Hd[i], Wd[i], xis[i], T, tol, power,
                              X=Xd[i] if want_X else None, A=Ad[i] if want_A else None,
                              resid_hist=hist[i] if want_hist else None,
                              omega=0.0 if omegas is None else float(omegas[i]))
             for i in range(n)]
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    iters = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    resid = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    beta = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    own = prec is None
    if own:
        prec = binding.Precoder(max_instances=max(n, 1), max_M=max(h.shape[0] for h in Hs),
                                max_K=max(h.shape[1] for h in Hs), variant=variant,
                                precision=precision, refine_sweeps=refine_sweeps,
                                refine_fp64=refine_fp64, simt_iteration=simt_iteration,
                                refine_tol=refine_tol, refine_solve_tol=refine_solve_tol,
                                refine_selective=refine_selective, refine_residual=refine_residual)
    try:
        if plan:
            p = prec.plan(insts, status, iters, resid, beta, use_graph=graph)
            for _ in range(repeats):
                binding.jacpcg_plan_execute(p, torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            binding.jacpcg_plan_destroy(p)
        else:
            for _ in range(repeats):
                prec.precode(insts, status, iters, resid, beta)
        torch.cuda.synchronize()
    finally:
        if own:
            prec.close()
    out = dict(
        W=[w.T.cpu().numpy().astype(np.complex128) for w in Wd],
        status=status.cpu().numpy(), iters=iters.cpu().numpy(), resid=resid.cpu().numpy(),
        beta=beta.cpu().numpy())
    if want_X:
        out["X"] = [x.T.cpu().numpy().astype(np.complex128) for x in Xd]
    if want_A:
        out["A"] = [a.T.cpu().numpy().astype(np.complex128) for a in Ad]
    if want_hist:
        out["hist"] = [h.cpu().numpy() for h in hist]
    return out
