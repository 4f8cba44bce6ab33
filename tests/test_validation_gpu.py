"""GPU validation: steady drag on a fixed sphere in a simple cubic array
against Hasimoto's dilute-array result; the error falls as the sphere spans
more lattice cells (the trend of the paper's fixed-sphere validation)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fixed_sphere_drag_converges_to_hasimoto():
    from paper_1011_2613_gb300 import validation as V

    res = [V.fixed_sphere_drag(R, relax=10.0) for R in (3.0, 4.5, 6.0)]
    errs = [abs(r["rel_error"]) for r in res]
    for r in res:
        assert abs(r["force_balance"]) < 1e-3  # steady: the sphere carries the whole body force
        assert abs(r["eps_volume"]) < 1e-12  # exact covered volume
        assert r["re_p"] < 0.25
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.04
