"""lee_energy_noalloc: the energy reduction for callers that cannot allocate
device memory (their fields sit in memory owned by another runtime or pool
that hands out pointers but allows no cudaMalloc).  It must agree with the
context-based lee_energy on the same field, on two calls in a row, using
only caller-owned inputs and outputs.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2609_24785_b300 import lee, workloads
from _helpers import make_solver

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-12}   # both reduce in FP64; only summation order differs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_noalloc_matches_context_energy(precision, cuda_device):
    import torch
    case = workloads.cylinder_pulse(256, nx=250, ny=190)
    s = make_solver(case, precision)
    s.step(40)
    s.sync()
    ref = s.energy()
    # the same field and node kinds, in caller-owned device memory (pitch = nx)
    dt = torch.float64 if precision == "fp64" else torch.float32
    p, u, v = (torch.from_numpy(s.field(f)).to(dt).to(cuda_device) for f in range(3))
    mask = torch.from_numpy(np.ascontiguousarray(s.mask())).to(cuda_device)
    out = torch.full((1,), -1.0, dtype=torch.float64, device=cuda_device)
    L = lee.load()
    stream = torch.cuda.current_stream(cuda_device)
    prec = lee.LEE_FP64 if precision == "fp64" else lee.LEE_FP32
    results = []
    for _ in range(2):
        rc = L.lee_energy_noalloc(C.c_void_p(p.data_ptr()), C.c_void_p(u.data_ptr()), C.c_void_p(v.data_ptr()),
                                  C.c_void_p(mask.data_ptr()), case.nx, case.ny, case.nx, prec, case.h,
                                  C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == lee.LEE_OK, L.lee_last_error(None)
        torch.cuda.synchronize()
        results.append(out.item())
    assert results[0] == results[1]                     # fixed summation order
    assert abs(results[0] - ref) <= TOL[precision] * ref, (results[0], ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_noalloc_skips_pitch_padding(precision, cuda_device):
    """Rows of `pitch` > nx elements: the padding columns (mask value 1 and
    large field values there) must not enter the sum."""
    import torch
    case = workloads.cylinder_pulse(256, nx=250, ny=190)
    s = make_solver(case, precision)
    s.step(40)
    s.sync()
    ref = s.energy()
    pitch = case.nx + 5
    dt = torch.float64 if precision == "fp64" else torch.float32

    def padded(a, fill):
        b = np.full((case.ny, pitch), fill, dtype=a.dtype)
        b[:, :case.nx] = a
        return b
    p, u, v = (torch.from_numpy(padded(s.field(f), 1e6)).to(dt).to(cuda_device) for f in range(3))
    mask = torch.from_numpy(padded(np.ascontiguousarray(s.mask()), 1)).to(cuda_device)
    out = torch.full((1,), -1.0, dtype=torch.float64, device=cuda_device)
    L = lee.load()
    stream = torch.cuda.current_stream(cuda_device)
    prec = lee.LEE_FP64 if precision == "fp64" else lee.LEE_FP32
    for _ in range(2):
        rc = L.lee_energy_noalloc(C.c_void_p(p.data_ptr()), C.c_void_p(u.data_ptr()), C.c_void_p(v.data_ptr()),
                                  C.c_void_p(mask.data_ptr()), case.nx, case.ny, pitch, prec, case.h,
                                  C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == lee.LEE_OK, L.lee_last_error(None)
        torch.cuda.synchronize()
        assert abs(out.item() - ref) <= TOL[precision] * ref, (out.item(), ref)


def test_energy_noalloc_rejects_rows_beyond_scratch(cuda_device):
    import torch
    L = lee.load()
    ny = 16385
    x = torch.zeros(8, dtype=torch.float64, device=cuda_device)
    rc = L.lee_energy_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()),
                              C.c_void_p(x.data_ptr()), 8, ny, 8, lee.LEE_FP64, 0.01, C.c_void_p(x.data_ptr()), None)
    assert rc == lee.LEE_ERR_ARG
    assert b"exceeds the static scratch" in L.lee_last_error(None)
