"""Helper run under torchrun by tests/test_slab_partition.py.

The y-slab partition of the left inverse, on CPU ranks (gloo).  Rank r holds only its
rows y0 <= y < y1 of the ensemble and of the right-hand sides.  It computes V1 (A_m^+ per
column, Gram route) for its columns, the x-pass of its rows, and its share of the y-sum
of V3, Sum_{y0 <= y < y1} b_{p_y}(y) (x-pass)[y, p_x], for the kept modes.  One all-reduce
(sum) of the K L partial sums per right-hand side follows, then the Delta_b^{-1/2}
scaling (V4).  V1 is independent per column (Sec. 3.10) and V3 is a sum over rows, so
the result must equal the whole-grid left inverse.  Rank 0 prints the relative error
against the oracle's whole-grid apply.
"""

import json
import os
import sys

import numpy as np
import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import basis, swift  # noqa: E402
from paper_2609_13327_b300 import synth  # noqa: E402

CASES = [synth.Workload("slab_wide", 16, 14, 3, 6, 3.0, 0.7, 3.0, 4, "fp64", 71),    # n_w < K
         synth.Workload("slab_tall", 16, 14, 6, 4, 3.0, 0.7, 3.0, 3, "fp64", 72)]    # n_w > K


def slab_rows(ny, world, rank):
    """Uneven contiguous slabs: the first ny % world ranks take one row more."""
    base, extra = divmod(ny, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def partial_sums(w, Z, x, lam, y0, y1):
    """This rank's share of V_b^T A^+ x, [R][K][L], from its rows only."""
    nx, ny = w.Nx, w.Ny
    cols = slice(y0 * nx, y1 * nx)
    Zs, xs = Z[:, :, cols], x[:, :, cols]                  # the rank's own data
    A = np.transpose(Zs, (2, 1, 0))                        # A_m [m][n_w][K]
    W, bad = swift.gram_route_pinv_apply(A, np.transpose(xs, (2, 1, 0)))
    assert bad < 0
    w_k = np.transpose(W, (2, 1, 0)).reshape(len(x), w.K, y1 - y0, nx)   # segments, this slab
    c = w_k @ basis.basis_1d(nx)                           # x-pass: [R][K][y][p_x]
    By = basis.basis_1d(ny)[y0:y1, :]                      # b_{p_y}(y) of the slab's rows
    part = np.einsum("yq,rkyp->rkqp", By, c)               # [R][K][p_y][p_x]
    S = basis.kept_modes(lam, w.tau)
    return part.reshape(len(x), w.K, ny * nx)[..., S], lam[S]


def main():
    dist.init_process_group("gloo")
    world, rank = dist.get_world_size(), dist.get_rank()
    out = []
    for w in CASES:
        Z = synth.ensemble(w)
        x = synth.rhs(w)
        lam = basis.spectrum_2d(w.Nx, w.Ny, w.ell_loc)
        y0, y1 = slab_rows(w.Ny, world, rank)
        part, lamS = partial_sums(w, Z, x, lam, y0, y1)
        t = torch.from_numpy(np.ascontiguousarray(part))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)           # K L values per right-hand side
        xt = t.numpy() / np.sqrt(lamS)
        ref = swift.apply_left_inverse(swift.Plan(Z, w.Nx, w.Ny, lam, w.tau), x)
        err = float(np.max(np.linalg.norm((xt - ref).reshape(len(x), -1), axis=1)
                           / np.linalg.norm(ref.reshape(len(x), -1), axis=1)))
        rows = [None] * world
        dist.all_gather_object(rows, (y0, y1))
        out.append({"case": w.name, "err": err, "rows": rows, "reduced_values": int(t.numel())})
    if rank == 0:
        sys.stdout.write("".join(json.dumps(o) + "\n" for o in out))
        sys.stdout.flush()
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
