"""The error path of the bounded waits in the tensor-core x-transform.

Every mbarrier wait of that kernel gives up after a fixed number of polls; the
thread block then waits for the loads and tensor-core work it had already
issued, frees its tensor memory and raises bit 1 of the plan's device flag,
which the host turns into PD_ERR_CUDA.  pd_debug_xform_timeout makes this
happen without any fault: the first thread block of the forward transform
issues none of its operand loads, so its consumers' waits (cut to 2^16 polls
for that launch) run out while nothing of that block is in flight.  The test
checks the status and message, and that the plan then gives the same
preconditioner as before the failure, bit for bit, and the oracle's within
the mixed-precision bound used by the preconditioner parity tests."""
import time
import zlib

import numpy as np
import pytest

import workloads as W
from helpers import EPS32, dev, host, lib_ready, make_plan, relerr
from oracle import closed_forms as CF
from oracle import operators as O
from oracle import paradiag as PD

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    return lib_ready()


def test_xform_wait_timeout_is_reported_and_plan_recovers(pd):
    import torch
    sp = W.Space(dim=2, nx=33, ny=20, nu=1e-2, ax=1.0, ay=0.5, bc_x=W.PERIODIC)
    pb = W.Problem(space=sp, nt=32, dt=1.0 / 32, scheme=W.CN, alpha=1e-3)
    r = W.uniform(W.SEED_BASE + zlib.crc32(b"xform_timeout") % 1000, pb.unknowns,
                  -1.0, 1.0).reshape(pb.nt, -1)
    plan = make_plan(pb, pd.PD_MIXED)
    rd = dev(r)
    z0 = host(plan.apply_precond(rd))

    zt = torch.empty_like(rd)
    t0 = time.perf_counter()
    st = pd.pd_debug_xform_timeout(plan.handle, pd._ptr(rd), pd._ptr(zt))
    elapsed = time.perf_counter() - t0
    print(f"XFORM_TIMEOUT status={st} seconds={elapsed:.3f} msg={pd.pd_last_error(plan.handle)!r}")
    assert st == pd.PD_ERR_CUDA
    assert "timed out" in pd.pd_last_error(plan.handle)

    # the plan (stream, tensor memory, flag) is usable again
    z1 = host(plan.apply_precond(rd))
    assert np.array_equal(z0, z1)
    zref = PD.precond_apply(pb, r)
    K = O.stencil(pb.space).toarray()
    l1, l2 = CF.lemma1_eigenvalues(pb)
    kap = max(np.linalg.cond(l1[k] * np.eye(K.shape[0]) + l2[k] * K) for k in range(pb.nt // 2 + 1))
    assert relerr(z1, zref) <= 2.0 * EPS32 * kap * (1.0 + np.log2(pb.nt)) / pb.alpha
    plan.close()


def test_xform_timeout_hook_needs_the_tensor_core_transform(pd):
    import torch
    sp = W.Space(dim=1, nx=31, nu=0.05)
    pb = W.Problem(space=sp, nt=16, dt=1.0 / 16, scheme=W.BE, alpha=1e-2)
    plan = make_plan(pb, pd.PD_MIXED)
    r = torch.zeros((pb.nt, 31), dtype=torch.float64, device="cuda")
    assert pd.pd_debug_xform_timeout(plan.handle, pd._ptr(r), pd._ptr(r)) == pd.PD_ERR_UNSUPPORTED
    plan.close()
