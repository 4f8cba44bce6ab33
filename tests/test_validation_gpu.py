"""GPU validation: steady drag on a fixed sphere in a simple cubic array (the
paper's fixed-sphere validation, Table 1: Re_p = 0.2 and 2, the error
falling as the sphere spans more lattice cells).

Re_p = 0.2 is compared with Hasimoto's dilute-array result (a Stokes-flow
closed form).  Re_p = 2 has no closed form (the paper compares with a
finite-volume code); there the check is the convergence itself: the drag
factor changes less with every refinement, and the flow's inertia raises it
above the Stokes value by an amount inside the range known for dilute
arrays."""
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


def test_fixed_sphere_finer_spheres():
    """d/l = 16, 24 and 32 (R = 8, 12, 16) in the FP32 deviation storage (the
    fixed-sphere drag agrees with FP64 to 1e-5 at R <= 8); R = 12 and 16 with
    the Eq. 6 covered fractions (the exact 3D rasteriser stops at R = 8): the
    error keeps falling."""
    from paper_1011_2613_gb300 import validation as V

    r8 = V.fixed_sphere_drag(8.0, relax=8.0, storage="f32dev")
    r12 = V.fixed_sphere_drag(12.0, relax=8.0, storage="f32dev", eps_method=1)
    r16 = V.fixed_sphere_drag(16.0, relax=8.0, storage="f32dev", eps_method=1)
    print(f"Re_p 0.2: K error R 8 {r8['rel_error']:.4f}, R 12 {r12['rel_error']:.4f}, R 16 {r16['rel_error']:.4f}")
    for r in (r8, r12, r16):
        assert abs(r["force_balance"]) < 2e-3
    assert abs(r16["rel_error"]) < abs(r12["rel_error"]) < abs(r8["rel_error"]) < 0.025


def test_fixed_sphere_re2_converges():
    """Re_p ~ 2 (the body force set for 2 by the Stokes estimate; the
    realised Re_p, 1.3-1.5, is lower by the inertial drag): successive
    refinements d/l = 6, 9, 12, 16 change K by less and less, and inertia
    raises K above its Re_p = 0.2 value at the same resolution (by about 1 %
    in this periodic array: the first inertial correction of an ordered
    array is of second order in Re)."""
    from paper_1011_2613_gb300 import validation as V

    Rs = (3.0, 4.5, 6.0, 8.0)
    hi = [V.fixed_sphere_drag(R, relax=8.0, re_p=2.0) for R in Rs]
    lo = [V.fixed_sphere_drag(R, relax=8.0, re_p=0.2) for R in Rs[:2]]
    K = [r["K"] for r in hi]
    steps = [abs(K[i + 1] - K[i]) / K[i + 1] for i in range(len(K) - 1)]
    print("Re_p 2: K", [round(k, 4) for k in K], "re_p", [round(r["re_p"], 3) for r in hi],
          "successive changes", [round(s, 4) for s in steps])
    for r in hi:
        assert abs(r["force_balance"]) < 2e-3
        assert 1.0 < r["re_p"] < 2.2
    assert steps[0] > steps[1] > steps[2]
    assert steps[2] < 0.03
    for a, b in zip(hi, lo):
        print(f"R {a['R']}: K(Re_p {a['re_p']:.2f}) / K(Re_p {b['re_p']:.2f}) = {a['K'] / b['K']:.4f}")
        assert 1.0 < a["K"] / b["K"] < 1.3
