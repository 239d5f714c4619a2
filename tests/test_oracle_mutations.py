"""Planted mistakes: each mutation of the oracle (made here, on the CPU, with monkeypatch) must make
at least one pin fail.  This shows the pins are sensitive to the plausible errors they target."""
import numpy as np
import pytest

from oracle import constraints as C, padmm as PA, rigid
import tests.test_oracle_constraints as TC
import tests.test_oracle_padmm as TP
import tests.test_oracle_rigid as TR


def _fails(fn, *a):
    try:
        fn(*a)
    except AssertionError:
        return True
    return False


def test_gyroscopic_sign_flip_is_caught(monkeypatch):
    orig = rigid.newton_euler_h

    def flipped(mass, inertia_diag, R, omega, gravity, force=None, torque=None):
        h = orig(mass, inertia_diag, R, omega, gravity, force, torque)
        Iw = R @ np.diag(inertia_diag) @ R.T
        h[3:] += 2 * np.cross(omega, Iw @ omega)
        return h

    monkeypatch.setattr(rigid, "newton_euler_h", flipped)
    import oracle.timestep as T
    monkeypatch.setattr(T, "newton_euler_h", flipped)
    assert _fails(TR.test_torque_free_symmetric_top_precession)


def test_dropped_lever_arm_is_caught(monkeypatch):
    orig = C.joint_rows

    def no_lever(jtype, parent, child, fp, fc, r, R):
        rows = orig(jtype, parent, child, fp, fc, r, R)
        out = []
        for k, (ba, Ja, bb, Jb, f) in enumerate(rows):
            if k < 3 and jtype != C.PRISMATIC:
                Jb = Jb.copy()
                Jb[3:] = 0.0
            out.append((ba, Ja, bb, Jb, f))
        return out

    monkeypatch.setattr(C, "joint_rows", no_lever)
    assert _fails(TC.test_joint_jacobian_is_derivative_of_error, C.REVOLUTE, False)


def test_wrong_cone_projection_is_caught(monkeypatch):
    def radial(x, n_bilateral, mu):            # scales onto the cone instead of projecting
        y = x.copy()
        for k, m in enumerate(mu):
            i = n_bilateral + 3 * k
            tn = np.hypot(x[i], x[i + 1])
            if tn > m * x[i + 2]:
                n = max(x[i + 2], 0.0)
                y[i:i + 2] = x[i:i + 2] * (m * n / tn if tn > 0 else 0.0)
                y[i + 2] = n
        return y

    monkeypatch.setattr(PA, "project_cone", radial)
    assert _fails(TP.test_cone_projection_kkt_and_brute_force, 0.3)


def test_transposed_desaxce_is_caught(monkeypatch):
    def on_tangent(v, n_bilateral, mu):        # correction put on a tangential row
        s = np.zeros_like(v)
        for k, m in enumerate(mu):
            i = n_bilateral + 3 * k
            s[i] = m * np.hypot(v[i], v[i + 1])
        return s

    monkeypatch.setattr(PA, "desaxce", on_tangent)
    assert _fails(TP.test_desaxce_operator)
