"""FP64 CPU oracle for the compressible semi-Lagrangian lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of the method (Spelten et al., "Supersonic shear and wall-bounded
flows with body-fitted meshes using the SLLBM", Sec. 3) written in numpy
float64.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library in
``paper_2412_09051_gb300``; the only shared module is ``workloads`` (seeded
input generators and plain configuration numbers, no method arithmetic).

Modules and the passage each follows:
  velocity_sets  Sec. 3.2 (cubature velocity sets, degree 9)
  equilibrium    Sec. 3.1, equilibrium Hermite expansion (N = 4) and g-equilibrium
  mesh           Sec. 3.1 Eq. (intf): cells with order-p Lagrange support points
  departure      Sec. 3.1 (departure point) and Sec. 3.3 (boundary schemes)
  step           Sec. 3.1 Eq. (1), moment definitions, Sec. 3.3 boundary schemes
  mlp            learned collision correction (not in the paper)

Parity status: the velocity sets, equilibrium, interpolation, inverse maps,
collision, thermal correction, forcing and mass rescaling are pinned by
closed forms, invariants and special cases (tests/test_oracle_*.py); the
temperature-dependent viscosity law of Sec. 4.3 by the shear-wave decay in
gas at T != T_ref (and per-node relaxation factors); the learned network's
forward pass and correction by a hand-evaluated one-path network; the
quasi-equilibrium term (Pr != 1) by its relaxation-rate invariants, the
Prandtl scaling of the compressible Couette temperature rise and the
thermal part of the sound attenuation.  The outlet scheme and the
equilibrium boundary are pinned by the far-field fixed point of a uniform
free stream (the population read, the boundary state) and geometrically
(mirrored source point); the bounce-back by its geometry (reflected source
point, opposite population) and, on flat walls, by the Couette profile.
The curved-wall bounce-back has no value pin beyond its geometry: "parity
partly unpinned" for that scheme.
"""
