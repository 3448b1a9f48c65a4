"""Small parity cases run against the bounds-check build of the library
(libdg_bounds.so: every computed cell, neighbour, tile and slab index is
checked on the device and a violation makes dg_check raise DG_ERR_BOUNDS).
Run as a script with DG_LIBRARY_VARIANT=bounds in the environment (see
test_gpu_bounds.py); every case must pass dg_check and match the oracle."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import workloads as W  # noqa: E402
from dg_helpers import assert_term_scale, dg_for, random_problem  # noqa: E402


def apply_cases():
    n = 0
    # generic kernels with one- and two-cell directions (the periodic
    # neighbour is the cell itself or the same cell on both sides)
    for dx, dv, k, cells in [(1, 1, 2, (1, 2)), (2, 1, 3, (2, 1, 3)), (2, 2, 2, (1, 2, 3, 1)),
                             (2, 3, 1, (2, 1, 1, 2, 3)), (3, 3, 1, (1, 2, 1, 2, 1, 3))]:
        for kind in ("const", "phase"):
            if kind == "phase" and dv < dx:
                continue
            dg, p = random_problem(dx, dv, k, cells, kind, seed=n)
            u = np.random.default_rng(n).standard_normal(p.n_dofs)
            for prec in (0, 1, 2):
                x = torch.tensor(u, device="cuda", dtype=torch.float32 if prec == 1 else torch.float64)
                xin = x.double().cpu().numpy()
                out = dg.apply(x, prec=prec)
                dg.check()
                assert_term_scale(out.double().cpu().numpy(), p.apply(xin), p.apply_abs(xin),
                                  1e-12 if prec == 0 else 1e-5, what=f"{dx}x{dv}v k{k} prec {prec}")
                wo = torch.empty_like(x)
                uu = torch.tensor(u, device="cuda")
                dg.rk_stage(x, wo, uu, 2, 1e-3, prec=prec)
                dg.check()
            dg.close()
            n += 1
    return n


def six_cases():
    n = 0
    # the specialised 6D kernels (64 and 128 threads per cell) on ragged
    # meshes with one- and two-cell directions
    for cells in [(1, 2, 1, 2, 1, 2), (2, 1, 2, 1, 2, 3), (2, 2, 2, 2, 2, 2)]:
        dg, p = random_problem(3, 3, 3, cells, "const", seed=len(cells) + sum(cells))
        assert dg.info.uniform_sides == 1
        u = np.random.default_rng(1).standard_normal(p.n_dofs)
        for prec in (1, 2):
            x = torch.tensor(u, device="cuda", dtype=torch.float32 if prec == 1 else torch.float64)
            xin = x.double().cpu().numpy()
            ref, scale = p.apply(xin), p.apply_abs(xin)
            for variant in (1, 2):
                dg.set_launch(prec, threads=128, cells_per_block=1, variant=variant)
                for adjoint in (False, True):
                    out = (dg.apply_adjoint if adjoint else dg.apply)(x, prec=prec)
                    dg.check()
                    if not adjoint:
                        assert_term_scale(out.double().cpu().numpy(), ref, scale, 1e-5,
                                          what=f"6D {cells} variant {variant}")
                wo = torch.empty_like(x)
                uu = torch.tensor(u, device="cuda")
                dg.rk_stage(x, wo, uu, 4, 1e-3, prec=prec)
                dg.check()
                n += 1
        dg.close()
    # the 6D workload's phase-space field, default launch, and its
    # host-buffer stage pipelined over v3 slabs (2, 6 and 10 cells along v3)
    for n3 in (2, 6, 10):
        dg, p = dg_for(W.shrink(W.config_6d(), cells_x=(2, 2, 2), cells_v=(2, 2, n3)))
        assert dg.info.uniform_sides == 1
        rng = np.random.default_rng(n3)
        u0 = torch.tensor(rng.standard_normal(dg.n_dofs))
        w_in = torch.tensor(rng.standard_normal(dg.n_dofs)).float()
        du, dw = u0.cuda(), w_in.cuda()
        dwo = torch.empty_like(dw)
        dg.rk_stage(dw, dwo, du, 1, 0.01, prec=1)
        dg.check()
        hu, hw = u0.clone().pin_memory(), w_in.clone().pin_memory()
        hwo = torch.empty_like(hw).pin_memory()
        dg.rk_stage_host(hw, hwo, hu, 1, 0.01, prec=1)
        torch.cuda.synchronize()
        dg.check()
        assert torch.equal(hu, du.cpu()) and torch.equal(hwo, dwo.cpu())
        # the delta-f stage (reference state: the stage vector's first half)
        dg.set_reference(du)
        uu = du.clone()
        dg.rk_step_df(uu, 1e-3, nsteps=1)
        dg.check()
        n += 1
        dg.close()
    # the Gauss-Lobatto collocation face-layer kernel
    from paper_2002_08110_gb300 import DG, basis_nodes
    w = W.shrink(W.config_6d(), cells_x=(2, 2, 2), cells_v=(2, 2, 2))
    nodes, qpts, _ = basis_nodes(1, w.k)
    dg = DG(e_nodes=W.e_table(w, qpts), basis=1, **W.dg_kwargs(w))
    x = W.separable_state(w, nodes, xp=torch, device="cuda")
    xf = x.float()
    out = dg.apply(xf, prec=1)
    wo = torch.empty_like(xf)
    dg.rk_stage(xf, wo, x.clone(), 0, 1e-3, prec=1)
    dg.check()
    assert torch.isfinite(out).all()
    dg.close()
    return n + 1


def four_and_batch_cases():
    from paper_2002_08110_gb300 import DG, DGBatch, reference_nodes
    n = 0
    for k, cells in [(1, (1, 2, 2, 1)), (3, (3, 2, 2, 3)), (5, (2, 1, 1, 2))]:
        w = W.shrink(W.config_4d(), cells_x=cells[:2], cells_v=cells[2:], k=k)
        dg, p = dg_for(w)
        u = np.random.default_rng(k).standard_normal(p.n_dofs)
        x = torch.tensor(u, device="cuda", dtype=torch.float32)
        xin = x.double().cpu().numpy()
        out = dg.apply(x, prec=1)
        dg.check()
        assert_term_scale(out.double().cpu().numpy(), p.apply(xin), p.apply_abs(xin), 1e-5,
                          what=f"4D k{k}")
        dg.close()
        n += 1
    ws = W.batched_instances(count=6, seed=3, cells_lo=1, cells_hi=4)
    dgs = [DG(**W.dg_kwargs(w)) for w in ws]
    batch = DGBatch(dgs)
    for prec in (0, 1):
        us = [torch.tensor(W.separable_state(w, reference_nodes(w.k)[0]), device="cuda") for w in ws]
        dt = torch.float32 if prec == 1 else torch.float64
        w0 = [torch.empty(w.n_dofs, device="cuda", dtype=dt) for w in ws]
        w1 = [torch.empty(w.n_dofs, device="cuda", dtype=dt) for w in ws]
        for t4 in (128, 256):
            batch.set_launch(512, 64, threads4=t4, order=3)
            batch.rk_step(us, w0, w1, [1e-3] * len(ws), nsteps=2, prec=prec)
            batch.check()
            n += 1
    batch.close()
    for dg in dgs:
        dg.close()
    return n


def main():
    from paper_2002_08110_gb300 import _lib
    assert _lib.LIB_PATH.endswith("libdg_bounds.so"), _lib.LIB_PATH
    n = apply_cases() + six_cases() + four_and_batch_cases()
    print(f"bounds-check build: {n} cases passed dg_check and the oracle comparison")


if __name__ == "__main__":
    main()
