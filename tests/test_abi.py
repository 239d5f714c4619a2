"""CPU-side checks of the C-ABI library: it loads, exports every function include/kamino.h declares,
and rejects bad world descriptions on the host before touching the GPU."""
import ctypes as C
import os

import numpy as np
import pytest

import worldgen as wg
from paper_2603_16536_gb300 import build as B
from paper_2603_16536_gb300 import kamino as K


@pytest.fixture(scope="module")
def lib():
    import os
    if not os.path.exists(B.LIB):
        B.build()
    return K.load_library()


def test_library_exports_every_declared_function(lib):
    names = K.header_functions()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layout_matches_header(tmp_path):
    """The ctypes mirror has the sizes and offsets the C compiler gives the header's structs (a probe
    compiled from include/kamino.h as plain C99)."""
    import shutil
    import subprocess
    assert K.ModelDesc.world_body_offset.offset == 8
    assert K.ModelDesc.gravity.offset == 8 + 15 * 8
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    probe = tmp_path / "probe.c"
    probe.write_text("""#include <stdio.h>
#include <stddef.h>
#include "kamino.h"
int main(void) {
    printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(kamino_solver_params), sizeof(kamino_model_desc),
           offsetof(kamino_model_desc, params), offsetof(kamino_model_desc, joint_drive),
           offsetof(kamino_model_desc, joint_limit), sizeof(kamino_model_info), sizeof(kamino_residual));
    return 0;
}
""")
    exe = tmp_path / "probe"
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I" + include, str(probe), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == [C.sizeof(K.SolverParams), C.sizeof(K.ModelDesc), K.ModelDesc.params.offset,
                   K.ModelDesc.joint_drive.offset, K.ModelDesc.joint_limit.offset, C.sizeof(K.ModelInfo),
                   K.RESIDUAL_DTYPE.itemsize]


def _create(ws, **override):
    m = K.Model.__new__(K.Model)
    try:
        K.Model.__init__(m, ws, **override)
    except K.KaminoError as e:
        return e.status, str(e)
    return 0, ""


def _mutated(fn):
    ws = wg.make_fourbar(num_worlds=2, seed=1)
    fn(ws)
    return ws


@pytest.mark.parametrize("mutate,status", [
    (lambda ws: ws.joint_parent.__setitem__(1, ws.joint_child[1]), 2),         # parent == child
    (lambda ws: ws.joint_child.__setitem__(0, 7), 2),                          # child out of range
    (lambda ws: ws.joint_type.__setitem__(2, 9), 2),                           # unknown joint type
    (lambda ws: ws.body_mass.__setitem__(0, 0.0), 2),                          # zero mass
    (lambda ws: ws.body_inertia.__setitem__((1, 2), -1.0), 2),                 # negative inertia
    (lambda ws: ws.joint_frame_parent.__setitem__((0, slice(3, 7)), 0.0), 2),  # null quaternion
    (lambda ws: ws.joint_actuator.__setitem__(0, 3), 2),                       # no such actuator slot
    (lambda ws: ws.world_mu.__setitem__(0, np.nan), 2),                        # bad friction
    (lambda ws: ws.joint_frame_child.__setitem__((1, 0), np.nan), 2),          # anchor not finite
    (lambda ws: ws.body_q0.__setitem__((2, 1), np.inf), 2),                    # initial pose not finite
    (lambda ws: ws.body_q0.__setitem__((0, slice(3, 7)), 0.0), 2),             # null initial quaternion
    (lambda ws: ws.body_u0.__setitem__((1, 4), np.nan), 2),                    # initial twist not finite
    (lambda ws: setattr(ws, "gravity", np.array([0.0, 0.0, np.inf])), 1),      # gravity not finite
])
def test_host_validation_rejects_bad_descriptions(lib, mutate, status):
    got, msg = _create(_mutated(mutate))
    assert got == status, msg
    assert lib.kamino_last_error().decode()


def test_non_finite_contact_point_is_rejected(lib):
    ws = wg.make_box(num_worlds=2)
    ws.contact_point[11, 2] = np.nan
    got, msg = _create(ws)
    assert got == 2 and "point not finite" in msg, msg


def test_bad_parameters_are_invalid_arg(lib):
    ws = wg.make_fourbar(num_worlds=1)
    for p in (K.make_params(rho=0.0), K.make_params(eta=-1.0), K.make_params(beta=2.0), K.make_params(warm_mode=7),
              K.make_params(residual_every=-1), K.make_params(residual_every=1025)):
        got, _ = _create(ws, params=p)
        assert got == 1


def test_oversized_world_is_unsupported(lib):
    # 70 contact candidates exceed the per-world candidate limit
    ws = wg.make_box()
    ws2 = wg.concat([ws] * 1)
    ws2.contact_body = np.zeros(70, np.int32)
    ws2.contact_point = np.zeros((70, 3))
    ws2.world_contact_offset = np.array([0, 70], np.int32)
    got, msg = _create(ws2)
    assert got == 7, msg


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.kamino_model_create(None, C.byref(h)) == 1
    assert lib.kamino_step(None, 1e-3, 10, 1e-6, None, None) == 1
    assert lib.kamino_state_free(None) == 0


def test_valid_model_needs_a_gpu(lib):
    """Without a CUDA device a valid description passes validation and fails with KAMINO_E_CUDA
    (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    got, msg = _create(wg.make_fourbar(num_worlds=2))
    assert got == 4, msg


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: without the compiled library the binding raises instead of computing."""
    from paper_2603_16536_gb300 import kamino
    saved = kamino._lib
    try:
        kamino._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            kamino.load_library(str(tmp_path / "libkamino_absent.so"))
    finally:
        kamino._lib = saved


@pytest.mark.parametrize("mutate,status", [
    (lambda ws: wg.with_joint_drives(ws, 2, 10.0, 1.0), 2),                   # not a KAMINO_DRIVE_* mode
    (lambda ws: wg.with_joint_drives(ws, wg.DRIVE_PD, -1.0, 1.0), 2),         # negative gain
    (lambda ws: wg.with_joint_drives(ws, wg.DRIVE_PD, np.inf, 1.0), 2),       # infinite gain
    (lambda ws: wg.with_joint_limits(ws, 1.0, -1.0), 2),                      # lower above upper
    (lambda ws: wg.with_joint_limits(ws, np.nan, 1.0), 2),                    # NaN bound
])
def test_model_rejects_bad_joint_dynamics(mutate, status):
    """Drive and limit descriptions are validated on the host before any GPU work."""
    got, msg = _create(mutate(wg.make_pendulum(actuated=True)))
    assert got == status, msg


def test_drives_and_limits_only_on_joint_coordinates():
    """Drives and limits act on the coordinate of a revolute or prismatic joint; a spherical joint
    with either is a topology error."""
    ws = wg.make_stewart(num_worlds=1, seed=0)
    sph = int(np.flatnonzero(ws.joint_type == wg.JOINT_SPHERICAL)[0])
    got, msg = _create(wg.with_joint_drives(ws, wg.DRIVE_TORQUE, armature=0.1, joints=[sph]))
    assert got == 2 and "drives" in msg, msg
    got, msg = _create(wg.with_joint_limits(ws, -0.5, 0.5, joints=[sph]))
    assert got == 2 and "limits" in msg, msg


def test_binding_checks_what_the_library_cannot():
    """Actuation tensors and host arrays are checked in the binding (the library sees raw pointers):
    a wrong element type, a non-contiguous or short buffer, or a CPU tensor raise ValueError."""
    import torch
    with pytest.raises(ValueError):
        K._tau_ptr(torch.zeros(24, dtype=torch.float32), torch.float32, 24)          # not on the GPU
    assert K._tau_ptr(None, torch.float32, 24) is None
    assert K._dev(None, torch.float32, "X") is None
    with pytest.raises(ValueError, match="X must be a contiguous CUDA"):
        K._dev(torch.zeros((4, 3)), torch.float32, "X", cols=3)                     # not on the GPU
    good = np.zeros(10, np.float32)
    assert K._host_ptr(K.BUF_BODY_Q, good, np.float32)[1] == 10
    for bad in (np.zeros(10, np.float64), np.zeros((10, 2), np.float32)[:, 0], [0.0] * 10):
        with pytest.raises(ValueError):
            K._host_ptr(K.BUF_BODY_Q, bad, np.float32)
    assert K._host_ptr(K.BUF_RESIDUAL, np.zeros(3, K.RESIDUAL_DTYPE), np.float32)[1] == 3
    with pytest.raises(ValueError):
        K._host_ptr(K.BUF_RESIDUAL, np.zeros(24, np.int32), np.float32)
