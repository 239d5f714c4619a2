"""Seeded synthetic world generators shared by the oracle, the tests and the benchmark.

This package only *describes* worlds: bodies (mass, principal inertia), joints (type, the two
bodies, a frame on each body), contact candidate points, the terrain and an initial state that
satisfies every joint exactly.  It contains none of the solver's arithmetic (no Jacobians, no
Delassus matrix, no time stepping); the CPU oracle and the CUDA path each implement those on
their own from the descriptions produced here.

Conventions (shared by every consumer of a ``WorldSet``):

* gravity acts along -z; the ground plane is z = 0 with normal +z;
* a body's frame sits at its centre of mass and is its principal frame, so its inertia is the
  diagonal ``body_inertia`` (kg m^2);
* body pose = (r[3], q[4]) with the quaternion stored (x, y, z, w); twist = (v[3], w[3]) with the
  angular velocity expressed in the world frame;
* a joint frame is (position[3], quaternion[4]) in the local frame of its body; its axes are
  e1, e2, e3.  Revolute: hinge about e3.  Prismatic: slide along e3.  Universal: free rotation
  about e1 of the parent frame and about e2 of the child frame.  Spherical: point joint.
  Fixed: weld.  ``joint_parent == -1`` attaches the joint to the world (frame given in world);
* ``joint_actuator`` is the slot of the joint in the world's actuation vector (torque about the
  hinge for a revolute, force along the slide for a prismatic), or -1 for a passive joint.
"""
from .worlds import (  # noqa: F401
    JOINT_REVOLUTE, JOINT_PRISMATIC, JOINT_UNIVERSAL, JOINT_SPHERICAL, JOINT_FIXED,
    JOINT_ROWS, TERRAIN_NONE, TERRAIN_PLANE, TERRAIN_HEIGHTFIELD, DRIVE_TORQUE, DRIVE_PD,
    WorldSet, concat, with_joint_drives, with_joint_limits, make_pendulum, make_free_body, make_box, make_fourbar, make_biped, make_biped_heightfield, make_biped_team,
    make_stewart, make_excavator, make_heightfield, actuation, count_loops,
)
