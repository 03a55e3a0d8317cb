"""FP64 CPU oracle for the voxel volume potential of the nested-mesh harmonic method.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of what the GPU library computes, written from the paper's equations
(Sections 2, 3 and 6 of "Accelerating frequency-domain numerical methods for weakly
nonlinear focused ultrasound using nested meshes").  Only the tests, the smoke
check and the CPU-baseline leg of the benchmark may import it; the product path
(the CUDA library and its Python binding) never does, and it shares no code,
table or constant generator with that path.  Inputs come from the seeded
generators in ``paper_2011_03009_gb300.synth``, which hold none of the method's
arithmetic.

Everything is complex128 / float64.  Modules:

- ``physics``   wavenumber of harmonic n (Eq. 2.2 with the power law), source
                coefficient of the truncated cascade (Eq. 2.6 folded with the sign of
                Eq. 3.2).
- ``greens``    Green's function (Eq. 3.3), the equal-volume-sphere self-cell integral
                and the voxel kernel lattice of the quadrature rule (Eq. 3.9).
- ``potential`` the discrete volume potential: brute-force double sum of Eq. 3.9 and
                the zero-padded circulant-embedding FFT evaluation (Section 3.1).
- ``cascade``   source terms f_n from products of lower harmonics (Eqs. 2.6, 3.5-3.8)
                and the nested-mesh harmonic loop (Section 6 algorithm).
- ``interp``    trilinear interpolation between nested voxel grids (Section 6).
- ``rayleigh``  incident field p1 as a monopole sum over bowl points (Eq. 3.10).

Parity pins: every function is checked by ``tests/test_oracle_*.py`` against
closed forms, brute force, invariants and the paper's printed constants.
"""
