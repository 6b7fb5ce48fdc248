"""The allocation-free mTPQ step (ftk_tpq_step_noalloc) against the regular
context path (ftk_tpq_step), two calls in a row. GPU only.

ftk_tpq_step_noalloc serves callers that cannot allocate device memory
(latency-bound loops that cannot take the synchronisation an allocation may
imply, processes whose device memory belongs to another framework's pool);
its reduction scratch is a static device array shared by all calls. This
file is collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest

from ftk_inputs import named, random_state

pytestmark = pytest.mark.gpu


def test_noalloc_step_matches_context_path():
    import torch
    from paper_1802_02854_gb300 import build
    build.build()
    import paper_1802_02854_gb300 as ftk

    for n, tile in [(12, 0), (16, 0)]:
        cl = named(n)
        K, J, ell = -1.0, 0.1, 0.5
        psi0 = random_state(n, 31 + n)
        ctx = ftk.Context(cl, K, J, "fp64", n_saved=1)
        ctx.set_state(psi0, ell)
        u_ref, _, h2_ref = ctx.tpq_step(2, 1000)
        psi = torch.from_numpy(psi0.copy()).cuda()
        out = torch.empty_like(psi)
        for k in range(2):                       # two calls in a row
            torch.cuda.synchronize()
            u, h2, q = ftk.ftk_tpq_step_noalloc(n, cl.bonds, K, J, ell, psi.data_ptr(), out.data_ptr())
            assert abs(u - u_ref[k]) <= 1e-12
            assert abs(h2 - h2_ref[k]) <= 1e-12 * max(1.0, abs(h2_ref[k]))
            psi = (out / q).contiguous()
        want = ctx.get_vector(0)
        got = psi.cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
        ctx.close()


def test_noalloc_rejects_oversize():
    from paper_1802_02854_gb300 import build
    build.build()
    import paper_1802_02854_gb300 as ftk

    cl = named(8)
    with pytest.raises(ftk.FtkError) as e:
        ftk.ftk_tpq_step_noalloc(31, cl.bonds, -1.0, 0.1, 0.5, 256, 512)
    assert e.value.status == ftk.FTK_EINVAL
    assert "FTK_NOALLOC_MAX_SITES" in str(e.value)


def test_noalloc_rejects_small_ell():
    """l below l_min = (1/N) sum_b lambda_max(h_b) is rejected as by
    ftk_tpq_init (l - H/N would not be positive semidefinite)."""
    import torch
    from paper_1802_02854_gb300 import build
    build.build()
    import paper_1802_02854_gb300 as ftk

    cl = named(8)
    psi = torch.from_numpy(random_state(8, 3)).cuda()
    out = torch.empty_like(psi)
    # K = -1, J = 0.1: l_min = (3/2) (1 + J) / 4 = 0.4125
    with pytest.raises(ftk.FtkError) as e:
        ftk.ftk_tpq_step_noalloc(8, cl.bonds, -1.0, 0.1, 0.40, psi.data_ptr(), out.data_ptr())
    assert e.value.status == ftk.FTK_EINVAL
    assert "l_min" in str(e.value)
    u, h2, q = ftk.ftk_tpq_step_noalloc(8, cl.bonds, -1.0, 0.1, 0.42, psi.data_ptr(), out.data_ptr())
    assert q > 0
