"""Plain, slow CPU oracle (FP64 numpy) of the sketched Tucker core update.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import, call or execute anything under this
directory; the CUDA library and its Python binding never do.  The oracle shares
no code with the CUDA path: the only module both consume is `synth`, which
draws the seeded inputs and holds none of the method's arithmetic.

Modules (each function cites the passage of the paper it restates):
  philox       Philox4x64-10 counter-based generator (Salmon et al. 2011)
  leverage     leverage and ridge leverage scores (Sec. 2, Eq. ridge_leverage_score_def)
  sampling     factored sampler, dedupe, probabilities, weights (Alg. 1, Alg. 3, Lemma 4.1)
  core_update  exact (Alg. 2 core line; Lemma 4.1 proof) and sketched (Alg. 3) core updates
  als          Alg. 2 factor updates, Tucker loss, RMSE
  adjoint      gradient of the frozen-sketch solve
  ridge_kron   lam-ridge scores of K by Lemma 4.1, d_eff(K), the overestimate constants of
               the sample count, and an exact sampler of l^lam(K) / d_eff(K)
  cp           regularised CP-ALS: exact and sketched factor updates on the Khatri-Rao
               design (Sec. 4's Khatri-Rao remark, Sec. 6's L2 extension)

Parity unpinned: none; every function has a pin in tests/test_oracle_*.py.
"""
from . import philox, leverage, sampling, core_update, als, adjoint, ridge_kron, cp  # noqa: F401
