"""Plain FP64 CPU oracle of the dual adaptive explicit monodomain scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run anything here.  The
product (the CUDA library and its Python binding) never calls into this
package, and this package never imports the product: the two share no code.
The only common dependency is the seeded input description in ``inputs/``,
which holds no arithmetic of the method.

Modules
-------
fem      finite-element assembly (bilinear quads, trilinear hexes, P1 tets),
         row-sum lumped mass, anisotropic conductivity tensor (Section 2,
         Section 3).
cells    cell models: Mitchell-Schaeffer, ten Tusscher-Panfilov 2006 and a
         test-only cubic bistable model; forward Euler / Rush-Larsen sub-steps.
scheme   Gershgorin stable step (Eq. 3), diffusion sub-step count l and reaction
         sub-step count k (Section 2), Strang splitting (Eq. 2), activation
         times, the OST / OSTAR / DAETI variants (Section 3).
metrics  normalised RMSE (Eq. 4), conduction velocity, aligned-AP difference.
adjoint  discrete adjoint of the split step for the Mitchell-Schaeffer model.

Parity status
-------------
Pinned (tests/test_oracle_*.py): assembly (closed-form element matrices,
linear/quadratic patch tests, printed dt_s of Section 3.1), Gershgorin bound
vs dense eigenvalues, diffusion sub-steps vs dense matrix powers and the
matrix exponential, conservation, the Strang/merge structure, the k and l
rules, Mitchell-Schaeffer fixed points / threshold / APD asymptote, the cubic
front speed, the adjoint (dot-product test and central differences).
TP06: parity unpinned against the TP06 publication itself (its equations are
not part of the paper); pinned by the thermal voltage from SI constants, the
reversal potential of every current (Nernst, GHK and exchanger zeros), the
pump half-saturation points, bounded monotone gates with positive time
constants, the published initial state being a resting state (fast gates at
steady state, net current balanced, 1000 ms unstimulated drift < 0.5 mV),
charge conservation, AP plausibility and fine-step self-convergence.  The
magnitudes of currents that vanish at rest (GNa, GKr, GKs, Gto, GpK) and the
SR/buffer constants are pinned only by AP plausibility.
"""
