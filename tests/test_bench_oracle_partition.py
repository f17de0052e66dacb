"""The reference arm's partitioned oracle run (bench.oracle_partitioned), on the CPU: the
blocks tile the element grid, and the result assembled from the blocks (each computed on
its own window with a three-element halo, in separate processes) equals the oracle's step
of the whole mesh."""
import numpy as np
import pytest

import bench
from helpers import Case, rel_l2


@pytest.mark.parametrize("nex,ney,nproc", [(96, 96, 16), (12, 8, 4), (7, 5, 3), (5, 5, 1)])
def test_blocks_tile_the_grid(nex, ney, nproc):
    bl = bench.oracle_blocks(nex, ney, nproc)
    assert len(bl) == nproc
    cover = np.zeros((ney, nex), dtype=int)
    for ex0, ex1, ey0, ey1 in bl:
        assert ex1 > ex0 and ey1 > ey0
        cover[ey0:ey1, ex0:ex1] += 1
    assert np.all(cover == 1)


def test_partitioned_step_equals_the_whole_mesh_step():
    from oracle import ark2
    nex, ney, nez, N, L, Lz = 12, 10, 2, 3, 60e3, 8e3
    case = Case(nex, ney, nez, N, L, L * ney / nex, Lz)
    dt = case.dt_for(15.0)
    q0 = case.state(77)
    sec, out, cols = bench.oracle_partitioned((nex, ney, nez, N, L, L * ney / nex, Lz), dt, q0,
                                              nproc=4, warmup=0, steps=1, timeout=600)
    ref = ark2.HEVI(case.mesh, case.col, dt).step(q0, 1)
    assert sec > 0 and cols > case.mesh.ncol
    e = rel_l2(out, ref)
    assert np.all(e <= 1e-13), e
