"""The domain decomposition's host side on the CPU with gloo ranks.

* the split of a lattice into time slabs and back, and the boundary bits of
  each slab (the time bit on the last slab only);
* the face exchange schedule (``dd.exchange_faces``) between 2 and 3 gloo
  ranks: every rank receives its upper neighbour's downward face and its lower
  neighbour's upward face, periodic in the rank index, also when both
  neighbours are the same rank;
* the decomposed hop on 2 gloo ranks with the oracle as the local hop: each
  rank hops its slab with the oracle (time wrapped inside the slab), packs
  its faces, exchanges them through ``dd.exchange_faces`` and replaces the
  wrapped time terms of its face sites -- the decomposition the GPU kernels
  implement, written out here in numpy -- and the assembled result equals the
  oracle's hop of the whole lattice.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2411_18511_gb300 import dd  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(target, world, *args):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=target, args=(r, world, port, out) + args) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        return dict(out)


def _init(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)


def test_slab_split_and_boundary_bits():
    dims = (12, 2, 4, 2)
    s = dd.TimeSlabs(dims, 3, bc=1 | 8)
    assert s.t_loc == 4 and s.v3 == 16
    assert [s.local(r).bc for r in range(3)] == [8, 8, 9]
    assert [tuple(s.local(r)) for r in range(3)] == [(4, 2, 4, 2)] * 3
    assert (s.lower(0), s.upper(2)) == (2, 0)
    q = synth.haar_links(dims, 1)
    psi = synth.gaussian_spinor(dims, 2, 2)
    parts = [s.split_spinor(psi, r) for r in range(3)]
    assert np.array_equal(s.join_spinor(parts), psi)
    # slab r holds the slices r*T_loc .. (r+1)*T_loc - 1 of every link direction
    V3 = 16
    for r in range(3):
        g = s.split_gauge(q, r)
        assert g.shape == (4, 4 * V3, 4)
        assert np.array_equal(g[:, 0], q[:, r * 4 * V3])
    for bad in ((8, 3), (12, 4), (6, 4)):
        with pytest.raises(ValueError):
            dd.TimeSlabs((bad[0], 2, 2, 2), bad[1])


def _exchange_rank(rank, world, port, out):
    _init(rank, world, port)
    try:
        n = 37
        to_lower = torch.full((n,), 1000.0 * rank + 1.0, dtype=torch.float64)
        to_upper = torch.full((n,), 1000.0 * rank + 2.0, dtype=torch.float64)
        from_upper = torch.zeros(n, dtype=torch.float64)
        from_lower = torch.zeros(n, dtype=torch.float64)
        dd.exchange_faces(to_lower, to_upper, from_upper, from_lower)
        out[rank] = (from_upper[0].item(), from_lower[0].item(), bool(torch.all(from_upper == from_upper[0])),
                     bool(torch.all(from_lower == from_lower[0])))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_schedule(world):
    res = _run(_exchange_rank, world)
    for r in range(world):
        up, down = (r + 1) % world, (r - 1) % world
        fu, fl, ok_u, ok_l = res[r]
        assert ok_u and ok_l
        assert fu == 1000.0 * up + 1.0     # the upper rank's downward face
        assert fl == 1000.0 * down + 2.0   # the lower rank's upward face


# ---- the decomposed hop with the oracle as the local hop --------------------

def _faces(slabs, rank, Lloc, psi_loc):
    """The rank's two faces as full 4-spinors (the GPU sends their two-spin
    projections, which carry the same information): (1 - g0) psi on t = 0, and
    (1 + g0) U_0(x)^+ psi(x) on t = T_loc - 1."""
    g0 = oracle.gamma(0)
    one = np.eye(4)
    v3 = slabs.v3
    nc = psi_loc.shape[-1]
    sl = psi_loc.reshape(slabs.t_loc, v3, 4, nc)
    down = np.einsum("ab,xbc->xac", one - g0, sl[0])
    U = Lloc.reshape(4, slabs.t_loc, v3, nc, nc)[0, -1]          # U_0 on the top slice
    Ud_psi = np.einsum("xdc,xbd->xbc", U.conj(), sl[-1])          # U^+ psi, colour index c
    up = np.einsum("ab,xbc->xac", one + g0, Ud_psi)
    return down, up


def _dd_rank(rank, world, port, out, dims, bc, seed):
    _init(rank, world, port)
    try:
        slabs = dd.TimeSlabs(dims, world, bc)
        q = synth.haar_links(dims, seed)
        psi = synth.gaussian_spinor(dims, 2, seed + 1)
        lat = slabs.local(rank)
        qloc = slabs.split_gauge(q, rank)
        Lloc = oracle.expand_links(lat, 2, qloc)
        if lat.bc & 1:  # the packed local links of the last slab carry the time boundary sign
            Lloc = Lloc.copy()
            Lloc.reshape(4, slabs.t_loc, slabs.v3, 2, 2)[0, -1] *= -1
        psi_loc = slabs.split_spinor(psi, rank)
        # the local hop, time wrapped inside the slab (the oracle; spatial signs as the local bits say)
        h = oracle.hop(lat, Lloc, psi_loc, bc=lat.bc & ~1)
        down, up = _faces(slabs, rank, Lloc, psi_loc)
        fu = torch.zeros(down.size * 2, dtype=torch.float64)
        fl = torch.zeros(up.size * 2, dtype=torch.float64)
        dd.exchange_faces(torch.from_numpy(down.view(np.float64).ravel().copy()),
                          torch.from_numpy(up.view(np.float64).ravel().copy()), fu, fl)
        from_upper = fu.numpy().view(np.complex128).reshape(down.shape)
        from_lower = fl.numpy().view(np.complex128).reshape(up.shape)
        # the wrapped terms the local hop added, and the remote ones that replace them
        wrong_down, wrong_up = _faces(slabs, rank, Lloc, psi_loc)
        hs = h.reshape(slabs.t_loc, slabs.v3, 4, 2)
        U_top = Lloc.reshape(4, slabs.t_loc, slabs.v3, 2, 2)[0, -1]
        # top slice: (1 - g0) U_0(x) psi(x + 0) with psi(x + 0) from the slab above
        hs[-1] += np.einsum("xcd,xad->xac", U_top, from_upper - wrong_down)
        # bottom slice: (1 + g0) U_0(x - 0)^+ psi(x - 0) from the slab below
        hs[0] += from_lower - wrong_up
        out[rank] = -0.5 * hs.reshape(h.shape)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("bc", [0, 1])
def test_decomposed_hop_on_two_gloo_ranks(bc):
    dims, seed = (8, 4, 2, 6), 421
    res = _run(_dd_rank, 2, dims, bc, seed)
    got = dd.TimeSlabs(dims, 2, bc).join_spinor([res[0], res[1]])
    q = synth.haar_links(dims, seed)
    psi = synth.gaussian_spinor(dims, 2, seed + 1)
    want = -0.5 * oracle.hop(dims, oracle.expand_links(dims, 2, q), psi, bc=bc)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)
