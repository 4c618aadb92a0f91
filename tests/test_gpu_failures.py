"""Failure paths under injected allocation failures (host side only).

The library routes every device and pinned-host allocation through one
function; with STK_FAIL_ALLOC_AFTER=N in the environment the first N
allocations succeed and the later ones fail as if the device were out of
memory.  For every N up to the number of allocations a setup + solve needs,
the calls must either succeed or return STK_ENOMEM, never crash, leave no
allocation behind once the problem is destroyed, and leave a problem that
solves correctly after the injector is switched off.
"""
import os

import numpy as np
import pytest

from seeded_inputs import manufactured_coefficients

pytestmark = pytest.mark.gpu

ENOMEM = -3


def _run(stk, n, k):
    import torch

    P = stk.StokesMG(n, k, 1.0, precision=stk.PREC_MIXED)
    try:
        b = torch.empty(P.layout()["n_total"], dtype=torch.float64, device="cuda")
        P.rhs(manufactured_coefficients(11), b)
        x = torch.zeros_like(b)
        info = P.solve(b, x, rtol=1e-8)
        return info
    finally:
        P.close()


@pytest.mark.parametrize("n,k", [(4, 2), (6, 1)])  # 2^3 and 3^3 coarse meshes
def test_every_allocation_failure_is_reported(stk, n, k):
    import torch

    _run(stk, n, k)  # kernels are loaded (and their device memory taken) on first use
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    outcomes = []
    try:
        for after in range(0, 40):
            os.environ["STK_FAIL_ALLOC_AFTER"] = str(after)
            try:
                info = _run(stk, n, k)
                outcomes.append("ok")
                assert info["converged"]
                break  # enough allocations succeed from here on
            except stk.StokesError as err:
                assert err.code == ENOMEM, str(err)
                outcomes.append("enomem")
    finally:
        os.environ.pop("STK_FAIL_ALLOC_AFTER", None)
    assert outcomes[0] == "enomem" and outcomes[-1] == "ok" and len(outcomes) > 5
    # nothing leaked: the device has the memory it had (to allocation granularity)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 64 * 2**20
    # and the library works normally again
    info = _run(stk, n, k)
    assert info["converged"] and info["relres"] <= 1e-8


def test_workspace_failure_then_retry(stk):
    """A smoothing call whose workspace allocation fails returns STK_ENOMEM;
    the same problem smooths correctly once memory is available again."""
    import torch

    from seeded_inputs import random_vector

    P = stk.StokesMG(4, 2, 1.0)
    N = P.layout()["n_total"]
    b = torch.from_numpy(random_vector(3, N)).cuda()
    x = torch.zeros_like(b)
    try:
        os.environ["STK_FAIL_ALLOC_AFTER"] = "1"  # the first workspace vector succeeds, the second fails
        with pytest.raises(stk.StokesError) as err:
            P.smooth(x, b)
        assert err.value.code == ENOMEM
    finally:
        os.environ.pop("STK_FAIL_ALLOC_AFTER", None)
    P.smooth(x, b)
    ref = torch.zeros_like(b)
    Q = stk.StokesMG(4, 2, 1.0)
    Q.smooth(ref, b)
    assert torch.equal(x, ref)
    P.close()
    Q.close()
