"""Oracle: a plain, slow, obviously-correct CPU implementation of the method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library (no kernels, headers, helpers, tables or generators); the only thing
both sides take from a common place is the seeded input description in the
``workloads`` package, which holds none of the method's arithmetic.

Everything is fp64.  Modules and the paper passages they follow:

* ``fock``        Fock-state words, sectors, hopping signs (Sec. "Exact
                  diagonalization"; state labels of App. D).
* ``hamiltonian`` the projected matrix H~_mn = <x~_m|H|x~_n> (Eq. (1) and the
                  Eq. defining the truncated-basis matrix), built explicitly.
* ``lanczos``     the Lanczos recursion of App. B and dense diagonalisation.
* ``sampler``     the Monte Carlo basis construction of Sec. "Subspace of the
                  ground state" with the acceptance probability of the
                  Boltzmann-factor Eq.; the random-number generator, the
                  ordering and the final-step truncation are not given by the
                  paper (parity of this part against the paper is unpinned:
                  it is pinned to the generator's published outputs,
                  acceptance statistics and structural invariants only).
"""
