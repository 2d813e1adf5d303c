"""FP64 CPU oracle for alternating-update NNCP (test infrastructure only).

This package is the plain, slow, obviously correct statement of what the GPU
hot path computes.  It exists to check the CUDA library and nothing else: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg
of ``bench.py`` may import it.  The product path (``paper_1909_01149_gb300``)
never imports, links or calls anything in here, and this package imports
nothing from the product path.

Everything is NumPy in float64.  The MTTKRP is computed by explicit
matricization times an explicit Khatri-Rao product, with no dimension tree, so
that a reader can check it against the definitions of the paper by eye.

Parity status per function (what pins it is in ``tests/test_oracle_*.py``):
  unfold, khatri_rao, mttkrp ........ pinned (brute-force sums, CP closed form,
                                      N=2 plain GEMM, two-stage 3-way equations)
  mttkrp_rows ....................... pinned (row-restricted brute-force sums,
                                      unsorted rows, every mode, N = 3..5)
  gram_hadamard ..................... pinned (explicit K^T K)
  nls_bpp ........................... pinned (scipy Lawson-Hanson NNLS,
                                      brute-force passive-set enumeration, KKT)
  nls_hals, nls_mu .................. pinned (objective non-increasing; HALS
                                      column step is the exact 1-D minimiser;
                                      HALS fixed point satisfies KKT)
  nls_admm .......................... pinned (uncapped ADMM reaches the BPP
                                      solution; hand-worked stop steps that
                                      separate the two ratios and their
                                      denominators; rho = 1 for S = 0)
  nls_pgd ........................... pinned (objective non-increasing; fixed
                                      point satisfies KKT)
  nls_ucp ........................... pinned (least squares on the explicit
                                      unfolding; ALS loss non-increasing;
                                      exact recovery of a noiseless CP tensor)
  nes_params ........................ pinned (closed forms for diagonal and
                                      rotated S; kappa cap)
  nls_nes ........................... pinned (uncapped: scipy NNLS of the plain
                                      and the proximal problem; the strongly
                                      convex accelerated rate bound; fixed
                                      point stops after one step)
  nes_extrapolate, model_error ...... pinned (explicit reconstruction of the
                                      extrapolated, projected model)
  normalize_columns ................. pinned (norms, reconstruction unchanged)
  fit_identity ...................... pinned (explicit reconstruction residual;
                                      alpha = 0 reports eps = 0)
  nncp .............................. pinned (noiseless planted tensor -> zero
                                      residual; monotone error for BPP/HALS)
  cp_loss_grad ...................... pinned (central finite differences)
"""

from .nncp import (  # noqa: F401
    unfold,
    khatri_rao,
    krp_except,
    mttkrp,
    mttkrp_rows,
    mttkrp_bruteforce,
    gram,
    gram_hadamard,
    nls_mu,
    nls_hals,
    nls_admm,
    nls_bpp,
    nls_bpp_row,
    nls_pgd,
    nls_ucp,
    nes_params,
    nls_nes,
    nes_extrapolate,
    model_error,
    NES_KAPPA,
    NES_MAX_INNER,
    NES_TOL,
    nls_objective,
    normalize_columns,
    cp_full,
    fit_identity,
    fit_explicit,
    sqnorm,
    nncp,
    cp_loss,
    cp_loss_grad,
    choose_split,
)
