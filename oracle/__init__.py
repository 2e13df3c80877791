"""Plain FP64 CPU oracle for known-pose, preconditioned-SGD cryo-EM refinement.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct
statement of what the CUDA path computes, written from Toader, Brubaker &
Lederman, arXiv 2311.16100 (Definition 2.1, Eqs. fwd model, optim cp,
hessian, hutch, diag est rule, thresh value, thresh, stochastic armijo and
Algorithm 1).  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the product path never does, and the
oracle shares no code with the CUDA path (only the seeded input generator in
``paper_2311_16100_gb300.synth`` feeds both).

Parity status per function (what pins it, see tests/test_oracle_pins.py):
  quat_to_rot          pinned: quaternion sandwich product, axis rotations
  nearest/trilinear    pinned: affine volumes (trilinear reproduces them
                       exactly), identity/90-degree rotations, brute-force
                       argmin over all grid points
  ctf                  pinned: textbook electron wavelengths, CTF zeros
  shift_phase          pinned: Fourier shift theorem (integer shifts = circular
                       roll of the real-space image), unitarity, and the
                       loss identity |x - C T S v| = |T* x - C S v|
  slice/adjoint        pinned: adjoint identity <Px, y> = <x, P*y>
  loss_grad            pinned: central finite differences (exact for a quadratic)
  hvp / dense H        pinned: linearity of the gradient, symmetry
  exact_diag           pinned: |Omega_j| + lam by brute-force counting,
                       diagonal of the dense Hessian, Proposition 3.1 bound
  splitmix64           pinned: published test vector
  hutchinson_diag      pinned: exact under nearest (Remark 3.3), unbiased
                       under trilinear (z-score against the dense Hessian)
  hutchinson_diag_at   pinned: equals hutchinson_diag at every voxel (the
                       same literal sum restricted to chosen rows)
  precomputed_preconditioner
                       pinned: brute-force pixel counts under nearest
                       (every probe exact, equal batches average to the
                       full diagonal), dense-Hessian z-scores under trilinear
  alpha_threshold      pinned: shell-ratio asymptotics, shell mean of diag(H)
  alg1_step            pinned: EM M-step equivalence (nearest, exact D, eta=1);
                       accepted eta against the closed-form Armijo bound;
                       preconditioner update in closed form under nearest
                       interpolation (every estimate exact, Remark 3.3):
                       D_avg^(k) = mean of the batch diagonals,
                       D^(k) = beta^k + (1 - beta^k) diag for equal batches;
                       the step v - eta g / max(|D|, alpha)
  coverage_features    pinned: nearest = brute-force pixel counts; the
                       weights of a pixel sum to 1 (sum = B n_px) and the
                       CTF^2 sum equals sum_i sum_p C_ip^2
  cg_solve             pinned: closed form under nearest interpolation
  lbfgs_solve          pinned: closed form under nearest interpolation, the
                       CG solution under trilinear interpolation with CTF, and
                       the quadratic's first-order condition H v = b
  diagnostics.fsc      pinned: Eq. fsc identities (1, -1, cos theta, shell
                       locality, energy partition), independent noise ~ 0
  diagnostics.shell_minmax / shell_index
                       pinned: integer shell rule, Legendre's three-square
                       theorem for the extremes of |k|^2 per shell
  diagnostics.condition_by_radius / p_ratio / kappa_lower_bound
                       pinned: brute-force max/min over the ball,
                       monotonicity, Eq. cond number p, Proposition 3.1
                       (unhit voxel => min = lam), p(R) ~ 3/(4R)
  mlp (learned preconditioner network; not in the paper)
                       pinned: BF16 rounding and GELU against torch's
                       library routines, backpropagation against central
                       finite differences of the FP64 network; features:
                       the |k| column voxel by voxel from its index
"""
from .geometry import (ball_mask, ctf_of_s2, ctf_pixels, default_r_max, disc_mask,
                       electron_wavelength_A, freq_axis, nearest_coords_fp32,
                       phase_shift, pixel_coords, quat_to_rot, sample_points, shift_phase,
                       stencil)
from .operators import (backproject_adjoint, coverage_features, dense_hessian,
                        exact_diag, hvp, loss, loss_grad, slice_project)
from .hutchinson import (hutchinson_diag, hutchinson_diag_at, probe_words, rademacher_probes,
                         splitmix64)
from .sgd import (alg1_step, alpha_threshold, cg_solve, full_rhs, lbfgs_solve,
                  precomputed_preconditioner, rel_err, shell_counts)
from . import diagnostics, mlp

__all__ = [n for n in dir() if not n.startswith("_")]
