"""CPU FP64 oracle for the skeletal-density complementarity score.

TEST INFRASTRUCTURE ONLY.  This package restates the paper's definitions
plainly and slowly so that the CUDA path can be checked against it.  Only the
test suite, the smoke check and the benchmark's CPU-baseline leg may import it;
the product path never does, and it imports nothing from the product package.

Modules
-------
sdf    Eq. 10A, 11, 12a, 13, 15, 16c, 17t: signed distance, membership and the SDF sum;
       the other phi-kernels of Section 4 (proximal, radial, skin/core).
score  Eq. 1 / Eq. 8: the pair-sum score of Gaussian-represented SDFs, its
       band-limited periodic form on the translation grid of Section 5, the
       per-rotation argmax and global top-k, and pose gradients.
refine Section 6: force and torque of the virtual energy E ~ -f, and the pose
       updates that climb the score (gradient ascent, conjugate gradient,
       damped rigid-body dynamics).
octree Section 5: adaptive tree sampling of the SDF, subdivided deepest where the
       skeletal density (the weight of a cell) is high.

Every function is pinned by tests under tests/ (closed forms, invariances,
brute force).  Absolute SDF and score values of the synthetic workloads have no
printed counterpart in the paper: parity unpinned beyond those checks.
"""
from . import octree, refine, score, sdf  # noqa: F401
