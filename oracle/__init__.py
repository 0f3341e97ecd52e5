"""Plain, slow FP64 CPU oracle of the MLS-MPM step and its gradient.

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import it. It shares
no code with the CUDA library (`paper_2303_02346_gb300`), and neither imports
the other; the seeded scene generators in `scenes` feed both.

Modules
-------
constitutive  corotated / von Mises / Drucker-Prager / liquid stress and
              return mappings with an SVD-based VJP (Sec. 3.2, Sec. 3.3, App. A)
tool          box SDF, soft Coulomb contact and tool kinematics (Sec. 3.2,
              Sec. 5.1, Sec. 4.2, App. B.1)
mpm           P2G, grid update, G2P, rollout and losses (Sec. 3.2, App. C)
rigid         particle-represented rigid bodies: shape-matching fit of a rigid
              motion after G2P and its enforcement (Sec. 3.2 "Rigid body")
sharing       gradient sharing between neighbouring particles and the
              attraction loss that approximates it (Sec. 5.1)
gas           grid-based incompressible gas after Stam 1999 (Sec. 3.2)
surrogate     3D convolutional neural operator over the grid (features from
              the particle state, BF16 rounding points of the CUDA kernels,
              forward, backward and Adam), imported by its tests on its own

Parity status: every function is pinned by tests in tests/test_oracle_*.py
(closed forms, conservation laws, affine reproduction, LAPACK, finite
differences, the paper's Table 5 constants); none is "parity unpinned".
"""
from . import constitutive, tool, rigid, mpm, sharing, gas  # noqa: F401
