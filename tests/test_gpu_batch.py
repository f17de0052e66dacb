"""The batching form: an ensemble of uneven members advanced by persistent launches and
CUDA graphs must give, for every member, exactly what a single-mesh context gives."""
import numpy as np
import pytest

from helpers import Case, rel_l2

pytestmark = pytest.mark.gpu

MEMBERS = [  # (nex, ney, nez, N, Lx, Ly, Lz)
    (3, 4, 2, 4, 90e3, 120e3, 10e3),
    (5, 2, 3, 5, 150e3, 60e3, 10e3),
    (2, 2, 4, 6, 60e3, 60e3, 12e3),
    (4, 3, 2, 5, 120e3, 90e3, 8e3),
    (1, 2, 3, 4, 30e3, 60e3, 9e3),
]


def _setup(C=15.0):
    import torch
    import paper_1702_04316_gb300 as pkg
    cases = [Case(*m[:3], m[3], *m[4:]) for m in MEMBERS]
    dts = [c.dt_for(C) for c in cases]
    b = pkg.Batch([m[:3] + m[4:] for m in MEMBERS], [m[3] for m in MEMBERS], dts)
    q = b.empty_state()
    for k, c in enumerate(cases):
        b.member(q, k).copy_(torch.from_numpy(c.state(100 + k, amp=0.5)))
    return pkg, torch, cases, dts, b, q


def test_batch_matches_single_contexts_exactly():
    pkg, torch, cases, dts, b, q = _setup()
    out = b.step_imex1d(q, b.empty_state(), 1)
    for k, (c, dt) in enumerate(zip(cases, dts)):
        nex, ney, nez, Lx, Ly, Lz, N = c.args
        g = pkg.Numa(nex, ney, nez, Lx, Ly, Lz, N, dt)
        ref = g.step_imex1d(b.member(q, k).contiguous(), g.empty_state(), 1)
        assert torch.equal(b.member(out, k), ref), k
        g.close()
    t = b.tuning()
    assert sorted(t) == [4, 5, 6]
    for v in t.values():
        assert v["rhs_threads_per_cta"] in (128, 256) and v["stage_columns_per_cta"] in (32, 64, 96)
        assert v["stage_threads_per_cta"] in (4 * v["stage_columns_per_cta"], 8 * v["stage_columns_per_cta"])


def test_graph_replay_equals_direct_launches_and_in_place():
    pkg, torch, cases, dts, b, q = _setup()
    a = b.step_imex1d(q, b.empty_state(), 3)
    b.set_graph(False)
    d = b.step_imex1d(q, b.empty_state(), 3)
    assert torch.equal(a, d)
    b.set_graph(True)
    qq = q.clone()
    b.step_imex1d(qq, None, 3)
    assert torch.equal(qq, a)


def test_batch_member_against_oracle():
    from oracle import ark2
    pkg, torch, cases, dts, b, q = _setup()
    out = b.step_imex1d(q, b.empty_state(), 1)
    for k in (0, 2):
        c = cases[k]
        q0 = b.member(q, k).cpu().numpy()
        ref = ark2.HEVI(c.mesh, c.col, dts[k]).step(q0, 1)
        e = rel_l2(b.member(out, k).cpu().numpy(), ref)
        assert np.all(e <= 1e-9), (k, e)


def test_batch_rejects_unsupported_order():
    import paper_1702_04316_gb300 as pkg
    with pytest.raises(pkg.NumaError):
        pkg.Batch([(2, 2, 2, 1e4, 1e4, 1e4)], [3], [1.0])
