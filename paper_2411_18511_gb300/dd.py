"""Domain decomposition of the lattice along time: the multi-GPU organisation
of the paper (Sec. 2.1.1 -- inner sites computed while the boundary data
travels -- and the scaling runs of Table 1), on the library's face calls.

* :class:`TimeSlabs` -- the split T = n T_loc (T_loc even): which slices a
  rank holds, its local lattice and boundary bits, and the host-side slicing
  of canonical fields into slabs and back (input preparation and assembly).
* :func:`exchange_faces` -- one hop's face exchange between the ranks of a
  ``torch.distributed`` group: ``to_lower`` goes to the rank below (arriving
  there as ``from_upper``), ``to_upper`` to the rank above (``from_lower``),
  periodic in the rank index, each received into the receiver's own buffer.
  NCCL on GPUs (no multicast, no peer memory handed to a kernel), gloo on the
  CPU for the tests.
* :class:`SlabHop` -- the even-odd hop D_{p,1-p} = -1/2 H of a decomposed
  lattice: per slab the face pack, the exchange (a device copy between slabs
  that share a GPU, or :func:`exchange_faces` between processes), the local
  hop with the tuned kernels meanwhile on the compute stream, and the
  boundary kernel once the faces have arrived.

Every arithmetic step runs in libhirep_gb300's kernels; this module only
moves bytes and orders launches.
"""

from __future__ import annotations

import numpy as np
import torch

from . import fields, hr


class TimeSlabs:
    """The lattice dims = (T, L1, L2, L3) split along time into n slabs."""

    def __init__(self, dims, n: int, bc: int = 0):
        dims = tuple(int(d) for d in dims)
        if n < 1 or dims[0] % n or (dims[0] // n) % 2:
            raise ValueError(f"T = {dims[0]} does not split into {n} slabs of an even number of slices")
        self.dims, self.n, self.bc = dims, int(n), int(bc)
        self.t_loc = dims[0] // n
        self.v3 = dims[1] * dims[2] * dims[3]

    def local(self, rank: int) -> hr.Lattice:
        """The local lattice of a rank: the time-boundary bit only on the last
        slab, which holds the global boundary slice; the spatial bits on all."""
        bc = (self.bc & ~1) | (self.bc & 1 if rank == self.n - 1 else 0)
        return hr.Lattice((self.t_loc,) + self.dims[1:], bc)

    def lower(self, rank: int) -> int:
        return (rank - 1) % self.n

    def upper(self, rank: int) -> int:
        return (rank + 1) % self.n

    def split_gauge(self, q: np.ndarray, rank: int) -> np.ndarray:
        """Canonical links [4, V, 4] -> the slab's [4, V_loc, 4]."""
        t0 = rank * self.t_loc
        return np.ascontiguousarray(q.reshape(4, self.dims[0], self.v3, 4)[:, t0:t0 + self.t_loc].reshape(4, -1, 4))

    def split_spinor(self, psi: np.ndarray, rank: int) -> np.ndarray:
        """Canonical spinor [V, 4, nc] -> the slab's [V_loc, 4, nc]."""
        t0 = rank * self.t_loc
        s = psi.reshape((self.dims[0], self.v3) + psi.shape[1:])[t0:t0 + self.t_loc]
        return np.ascontiguousarray(s.reshape((-1,) + psi.shape[1:]))

    def join_spinor(self, parts) -> np.ndarray:
        """The slabs' canonical spinors back into the global one."""
        return np.concatenate([np.asarray(p) for p in parts], axis=0)


def exchange_faces(to_lower: torch.Tensor, to_upper: torch.Tensor, from_upper: torch.Tensor,
                   from_lower: torch.Tensor, group=None, wait: bool = True):
    """Send to_lower to the rank below and to_upper to the rank above, and
    receive from_upper (the upper rank's to_lower) and from_lower (the lower
    rank's to_upper), periodic in the rank index.  The four operations are
    issued in one batch in a fixed order -- send down, send up, receive from
    above, receive from below -- with tags 0 (downward) and 1 (upward): with
    two ranks both neighbours are the same process, and the order (NCCL) or
    the tags (gloo) keep the two messages apart.  wait=False returns the
    pending requests instead of waiting for them (their wait() makes the
    current stream wait on NCCL, so kernels issued before it overlap)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if world == 1:
        from_upper.copy_(to_lower)
        from_lower.copy_(to_upper)
        return []
    down = dist.get_global_rank(group, (rank - 1) % world) if group is not None else (rank - 1) % world
    up = dist.get_global_rank(group, (rank + 1) % world) if group is not None else (rank + 1) % world
    ops = [dist.P2POp(dist.isend, to_lower, down, group, 0),
           dist.P2POp(dist.isend, to_upper, up, group, 1),
           dist.P2POp(dist.irecv, from_upper, up, group, 0),
           dist.P2POp(dist.irecv, from_lower, down, group, 1)]
    works = dist.batch_isend_irecv(ops)
    if wait:
        for w in works:
            w.wait()
        return []
    return works


class SlabHop:
    """The even-odd hop of a lattice split into slabs that live on this
    process's GPU (every slab of the lattice: the one-GPU form of the
    multi-GPU data flow), packed in precision prec of representation rep."""

    def __init__(self, ctx: hr.Context, slabs: TimeSlabs, rep: int, prec: int, q: np.ndarray):
        self.ctx, self.slabs, self.rep, self.prec = ctx, slabs, rep, prec
        self.gauge = [fields.pack_gauge(ctx, slabs.local(r), rep, prec, fields.gauge_to_device(slabs.split_gauge(q, r)))
                      for r in range(slabs.n)]
        fb = hr.hr_dd_face_bytes(slabs.local(0), rep, prec)
        mk = lambda: [fields.empty_bytes(fb) for _ in range(slabs.n)]  # noqa: E731
        self.to_lower, self.to_upper, self.from_upper, self.from_lower = mk(), mk(), mk(), mk()
        self.comm = torch.cuda.Stream()

    def pack_input(self, psi: np.ndarray, in_parity: int):
        """The slabs' packed input fields (sites of in_parity) from a global canonical spinor."""
        return [fields.pack_spinor(self.ctx, self.slabs.local(r), self.rep, self.prec, in_parity,
                                   fields.spinor_to_device(self.slabs.split_spinor(psi, r)))
                for r in range(self.slabs.n)]

    def apply(self, out_parity: int, src, out):
        """out[r] = D_{p,1-p} src[r] on every slab (packed local fields):
        faces packed, exchanged by device copies on the comm stream while the
        local hops run on the current stream, then the boundary kernels."""
        S, ctx, rep, prec = self.slabs, self.ctx, self.rep, self.prec
        compute = torch.cuda.current_stream()
        for r in range(S.n):
            hr.hr_dd_pack_faces(ctx, S.local(r), rep, prec, 1 - out_parity, self.gauge[r], src[r],
                                self.to_lower[r], self.to_upper[r], compute)
        packed = torch.cuda.Event()
        packed.record(compute)
        self.comm.wait_event(packed)
        with torch.cuda.stream(self.comm):
            for r in range(S.n):
                self.from_upper[S.lower(r)].copy_(self.to_lower[r], non_blocking=True)
                self.from_lower[S.upper(r)].copy_(self.to_upper[r], non_blocking=True)
        arrived = torch.cuda.Event()
        arrived.record(self.comm)
        for r in range(S.n):  # the inner sites need nothing remote
            hr.hr_dirac_eo(ctx, S.local(r), 0.0, rep, prec, out_parity, hr.HR_OP_HOP, 1, self.gauge[r], src[r],
                           out[r], None, compute)
        compute.wait_event(arrived)
        for r in range(S.n):
            hr.hr_dd_hop_boundary(ctx, S.local(r), rep, prec, out_parity, self.gauge[r], src[r],
                                  self.from_lower[r], self.from_upper[r], out[r], compute)

    def hop(self, out_parity: int, psi: np.ndarray) -> np.ndarray:
        """Global canonical in, global canonical out (sites of out_parity; the rest zero)."""
        S = self.slabs
        src = self.pack_input(psi, 1 - out_parity)
        out = [fields.empty_spinor(S.local(r), self.rep, self.prec, out_parity) for r in range(S.n)]
        self.apply(out_parity, src, out)
        return S.join_spinor([fields.unpack_spinor(self.ctx, S.local(r), self.rep, self.prec, out_parity,
                                                   out[r]).cpu().numpy() for r in range(S.n)])


def rank_hop(ctx: hr.Context, slabs: TimeSlabs, rank: int, rep: int, prec: int, out_parity: int, gauge, src, out,
             faces, group=None):
    """One rank's share of the hop when every rank is a process with its own
    GPU: pack, exchange over the process group (NCCL send / receive into this
    rank's own buffers), the local hop, the boundary.  faces: four device
    buffers (to_lower, to_upper, from_upper, from_lower) of hr_dd_face_bytes.
    The exchange is posted right after the pack and the local hop is issued
    before waiting for it, so the inner sites run while the faces travel."""
    lat = slabs.local(rank)
    to_lower, to_upper, from_upper, from_lower = faces
    hr.hr_dd_pack_faces(ctx, lat, rep, prec, 1 - out_parity, gauge, src, to_lower, to_upper)
    works = exchange_faces(to_lower, to_upper, from_upper, from_lower, group, wait=False)
    hr.hr_dirac_eo(ctx, lat, 0.0, rep, prec, out_parity, hr.HR_OP_HOP, 1, gauge, src, out)
    for w in works:
        w.wait()
    hr.hr_dd_hop_boundary(ctx, lat, rep, prec, out_parity, gauge, src, from_lower, from_upper, out)
