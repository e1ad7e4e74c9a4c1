"""FP64 CPU oracle of the adjoint Lattice Boltzmann hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never calls it and
shares no code with it.

The oracle is plain PyTorch CPU code in float64:

* ``lattice``  - velocity sets (Sec. 3 list e1..e19, D3Q7 = e1..e7, D2Q9 =
  the z = 0 members), weights, opposite directions and the MRT moment bases.
* ``model``    - node types, the local collision operator W^x of Eq.
  "normal:iteration" for every node type (FMRT/BGK with Exact-Difference
  forcing and Darcy porosity, bounce-back, Zou-He, passive scalars) and the
  node-local objectives F^x of Eq. "objective:function".
* ``solver``   - the periodic streaming of Sec. 2.1 in the paper's push form,
  the primal iteration, the unsteady discrete adjoint (the time-dependent
  form of Eqs. "adjoint:iteration"/"adjoint:operator" with the gradient of
  Eq. "adjoint:derivative" accumulated over the steps), the frozen-state
  ALBS mode, the one-shot optimisation of Sec. 3.3 with the penalty of
  Eq. P and the threshold scan of Sec. 3.2, the MMA design loop of
  Sec. 3.3, and a central finite-difference driver.
* ``mma``      - the Method of Moving Asymptotes (Svanberg's method, which
  Sec. 3.3 cites without formulas) for box-bounded design variables.

The adjoint collision is the vector-Jacobian product of W^x, taken by
PyTorch's reverse-mode autodiff (a library primitive, in the role TAPENADE
plays in Sec. 3.4); the CUDA path instead carries a hand-derived transpose.

Pins (``tests/test_oracle_*.py``, run with ``-m "not gpu"``): lattice
isotropy, MRT orthogonality and the T = omega I reduction to BGK, Lemma 1,
mass/momentum conservation, the Poiseuille closed form, Zou-He prescribed
values, Exact-Difference forcing, porosity limits, scalar diffusion decay,
the one-step duality identity and central finite differences of J.
"""
