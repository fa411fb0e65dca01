"""Failure detection on the GPU without a fault: a bounded device wait that
runs out (an mbarrier nothing arrives at) must come back to the host as
LAMINO_ETIMEOUT from the status check, clear on reading, leave other plans
untouched and leave the context usable (the same results as before)."""
import math

import pytest
import torch

from paper_2401_11101_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ETIMEOUT, EINVAL = -4, -1


@pytest.fixture(scope="module")
def L():
    from paper_2401_11101_gb300 import _build, lamino
    _build.build()
    lamino.load_library()
    return lamino


def test_expired_wait_reports_timeout_and_context_survives(L):
    g = I.Geometry(16, 16, 8, 12, 10, 26, math.radians(25.0))
    q = torch.as_tensor(I.random_projections(g, 41), dtype=torch.float32).cuda()
    with L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt) as p, \
            L.Plan(g.n0, g.n1, g.n2, g.nproj, g.det_w, g.det_h, g.tilt) as other:
        ref_d = p.backproject(q, "direct").cpu()
        ref_f = p.backproject(q, "fourier").cpu()
        p.status()
        p.selftest_wait(200_000)                 # gives up after 0.2 s
        with pytest.raises(L.LaminoError) as e:
            p.status()
        assert e.value.code == ETIMEOUT
        assert "bounded device wait" in str(e.value)
        p.status()                               # the flag was cleared
        other.status()                           # error words are per plan
        assert torch.equal(p.backproject(q, "direct").cpu(), ref_d)
        assert torch.equal(p.backproject(q, "fourier").cpu(), ref_f)
        p.status()
        for bad in (0, 5_000_001):
            with pytest.raises(L.LaminoError) as e:
                p.selftest_wait(bad)
            assert e.value.code == EINVAL
