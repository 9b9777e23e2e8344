"""Plain CPU oracle for the reduced-order (PODP "Matrix Method") MPT path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import or execute anything in
this package.  The CUDA library never calls it, and this package imports
nothing from the CUDA library or its Python binding.  Inputs come from the
seeded generators in ``workloads/``.

Everything is float64 / complex128 numpy + scipy, written step by step in the
order and notation of the paper (Elgy & Ledger, "Efficient Computation of
Magnetic Polarizability Tensor Spectral Signatures for Object
Characterisation in Metal Detection"):

* ``fom``        full-order solves (Eq. (9)) and the Full Matrix Method tensors
                 R (Eq. (11)) and I (Eq. (12)) with the same-basis
                 simplification of Remark 3.1;
* ``tsvd``       snapshot SVD and truncation (Sect. 4.1, Eqs. (13)-(15));
* ``rom``        Galerkin projection (Eq. (17)) and the Matrix Method tensors
                 (Eqs. (18), (19));
* ``certificate`` the a-posteriori certificate of Lemma 4.2 (Eq. (20));
* ``adapt``      the adaptive snapshot loop of Algorithm 1;
* ``grads``      derivatives of R and I with respect to omega, a conductivity
                 scale and a permeability scale (forward mode, dense);
* ``pencil``     an independent second sweep path through the generalized
                 Hermitian eigenproblem of the reduced pencil.

Pins: every function is checked in ``tests/test_oracle_*.py`` against facts
the paper or the mathematics fix (symmetry, Galerkin exactness at the
snapshots, energy identities, limits, scaling laws, brute force).  Functions
without such a pin are marked "parity unpinned" in their docstring.
"""
from . import fom, tsvd, rom, certificate, pipeline, adapt, grads, pencil  # noqa: F401
