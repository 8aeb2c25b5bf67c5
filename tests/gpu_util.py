"""Helpers for the GPU parity tests (marshalling only)."""
import numpy as np
import torch

import graphgen as gg

DEV = torch.device("cuda:0")


def to_dev(g: gg.DenseGraph) -> torch.Tensor:
    rows = g.rows if g.rows.size else np.zeros((max(g.n, 1), max(g.words, 1)), np.uint32)
    return torch.from_numpy(np.ascontiguousarray(rows).view(np.int32)).to(DEV)


def run_dense(ctx, g: gg.DenseGraph):
    from paper_1508_06329_gb300 import binding as B
    rows = to_dev(g)
    res = torch.full((4,), -7, dtype=torch.int32, device=DEV)
    order = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device=DEV)
    B.chordal_test_dense(ctx, rows, g.n, res, order)
    torch.cuda.synchronize()
    return tuple(res.cpu().tolist()), order[:g.n].cpu().numpy()
