"""Device-buffer helpers around the C ABI: allocate packed fields as torch byte
tensors and move canonical fields in and out of the packed layouts.

Only allocation and marshalling happen here; layout conversion runs in the
library's pack/unpack kernels.
"""

from __future__ import annotations

import numpy as np
import torch

from . import hr


def nc_of(rep: int) -> int:
    return 2 if rep == hr.HR_FUND else 3


def volume(dims) -> int:
    v = 1
    for d in dims:
        v *= int(d)
    return v


def empty_bytes(nbytes: int, device="cuda") -> torch.Tensor:
    """A 256-byte aligned device byte buffer (torch's caching allocator aligns to 512)."""
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def gauge_to_device(q, device="cuda") -> torch.Tensor:
    """Canonical gauge double[4][V][4] on the device."""
    t = torch.as_tensor(np.ascontiguousarray(q, dtype=np.float64))
    return t.to(device).contiguous()


def spinor_to_device(psi, device="cuda") -> torch.Tensor:
    """Canonical spinor(s) complex[(n,) V, 4, nc] -> device complex128 tensor."""
    t = torch.as_tensor(np.ascontiguousarray(psi, dtype=np.complex128))
    return t.to(device).contiguous()


def pack_gauge(ctx, dims, rep, prec, q_dev, stream=None) -> torch.Tensor:
    out = empty_bytes(hr.hr_gauge_packed_bytes(dims, rep, prec), q_dev.device)
    hr.hr_gauge_pack(ctx, dims, rep, prec, q_dev, out, stream)
    return out


def build_clover(ctx, dims, rep, prec, kind, m0, c_sw, q_dev, stream=None) -> torch.Tensor:
    """Packed clover field (hr_clover_build) from canonical device links."""
    out = empty_bytes(hr.hr_clover_packed_bytes(dims, rep, prec), q_dev.device)
    hr.hr_clover_build(ctx, dims, rep, prec, kind, m0, c_sw, q_dev, out, stream)
    return out


def pack_spinor(ctx, dims, rep, prec, parity, psi_dev, stream=None) -> torch.Tensor:
    """psi_dev: complex128 [V,4,nc] or [n_rhs,V,4,nc] (canonical, on the device)."""
    n_rhs = 1 if psi_dev.dim() == 3 else psi_dev.shape[0]
    out = empty_bytes(hr.hr_spinor_packed_bytes(dims, rep, prec, parity, n_rhs), psi_dev.device)
    hr.hr_spinor_pack(ctx, dims, rep, prec, parity, n_rhs, torch.view_as_real(psi_dev), out, stream)
    return out


def unpack_spinor(ctx, dims, rep, prec, parity, packed, n_rhs: int = 1, stream=None) -> torch.Tensor:
    """Packed -> canonical complex128 [V,4,nc] (or [n_rhs,...]); other-parity sites are zero."""
    V = volume(dims)
    shape = (V, 4, nc_of(rep)) if n_rhs == 1 else (n_rhs, V, 4, nc_of(rep))
    out = torch.zeros(shape, dtype=torch.complex128, device=packed.device)
    hr.hr_spinor_unpack(ctx, dims, rep, prec, parity, n_rhs, packed, torch.view_as_real(out), stream)
    return out


def empty_spinor(dims, rep, prec, parity, n_rhs: int = 1, device="cuda") -> torch.Tensor:
    return empty_bytes(hr.hr_spinor_packed_bytes(dims, rep, prec, parity, n_rhs), device)


def zeros_spinor(dims, rep, prec, parity, n_rhs: int = 1, device="cuda") -> torch.Tensor:
    return torch.zeros(max(hr.hr_spinor_packed_bytes(dims, rep, prec, parity, n_rhs), 1),
                       dtype=torch.uint8, device=device)
