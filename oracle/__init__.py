"""FP64 CPU oracle for shape-constrained gravitational registration.

TEST INFRASTRUCTURE.  This package is the slow, plain reference that the CUDA
library is checked against.  Only the test-suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.
The CUDA path never imports, links or calls anything here, and this package
shares no code with it; the only thing both sides use is the seeded input
generator ``paper_1902_01061_gb300.synth``, which holds none of the method's
arithmetic.

Everything follows the paper (Agarwal & Bhowmick, "3D Point Cloud
Registration with Shape Constraint", arXiv 1902.01061) step by step, in
float64, with library primitives (sort, eigvalsh, SVD) standing in for the
textbook operations the paper names.  Where the paper is silent or garbled the
reading taken is stated next to the code (readings R1..R14).

Functions and their pins (the tests under ``tests/test_oracle_*.py``):

* ``knn``            - R1 exact float32 key; pinned to a pure-Python scalar
                       brute force and an exact-shift invariance.
* ``curvature``      - Sec. III-A / IV; pinned to hand cases (plane, line,
                       axis star = 1/3, box corners = 1/14) and invariances.
* ``curvature_radius`` - the radius neighbourhood of Sec. IV; pinned to the
                       same hand cases (plane, axis star) and to the k-nearest
                       curvature when the radius neighbourhood is the whole
                       cloud.
* ``register_pyramid`` - the pyramidal schedule of Sec. IV; pinned to
                       ``register`` for a single level, for two equal levels
                       (template and Eq. 12 position carried over), for a
                       sigma scale (times the reference std), and to one
                       method step with a second level's own descriptors.
* ``nearest`` / ``change_mask`` - the change-detection post-pass; pinned to
                       the scalar brute force of the kNN pins (k = 1).
* ``sigma_auto``     - R3; pinned to a closed form (two-valued population).
* ``forces``         - Eq. 5 with Eq. 3, 10, 11; pinned to the two-point hand
                       case, the p=1 closed forms, Newton's third law,
                       rotation/translation equivariance and scaling.
* ``force_row_magnitudes`` - per-row sums of term magnitudes of Eq. 5 (the
                       condition number of each force sum); pinned to hand
                       cases (one pull: kappa = 1; balanced pulls: f = 0) and
                       to the Euclidean norm of an explicit term list.
* ``potential`` / ``potential_grad`` - the potential whose negative gradient is
                       Eq. 5; pinned by central finite differences.
* ``force_vjp``      - the force field's vector-Jacobian product; pinned by
                       central differences of ``forces``.
* ``g_schedule``     - Eq. 12; pinned to its closed-form values.
* ``kabsch``         - Eq. 6; pinned to exact recovery of a known rotation,
                       including the reflection case.
* ``scale_factor``   - Sec. III-B / Eq. 8 with R8; pinned to one-step recovery
                       of a scaled copy.
* ``partial_sums`` / ``update_from_totals`` - the iteration split at the
                       13 totals (for row sharding); pinned to ``step_once``.
* ``register``       - the whole iteration (Eq. 5-12); pinned to the fixed
                       point at the aligned pose and to recovery of known
                       synthetic transforms.
* ``register_from_partials`` - ``register`` with each iteration's totals
                       added from row blocks (so a process pool can share the
                       force pass); pinned to ``register``.
"""
from .scgr_oracle import (  # noqa: F401
    Params,
    knn,
    curvature,
    sigma_auto,
    cloud_stats,
    descriptors,
    forces,
    forces_rows,
    force_row_magnitudes,
    potential,
    potential_grad,
    pose_potential_and_grad,
    rodrigues,
    g_schedule,
    kabsch,
    scale_factor,
    polar,
    register,
    register_from_partials,
    step_once,
    partial_sums,
    update_from_totals,
    curvature_radius,
    register_pyramid,
    nearest,
    change_mask,
    force_vjp,
)
