"""Plain, slow, FP64 CPU oracle for the localized Hamiltonian application and the
sparse H_ab / S_ab build of the Daubechies-wavelet linear-scaling DFT method
(arXiv 1401.7441).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or
execute anything under ``oracle/``; only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle shares no code with the GPU library (``paper_1401_7441_gb300``): it has
its own filter derivation (``filters.py``, multi-precision, written out once to
``filters_d16.txt``), its own locreg geometry and segment keys (``geometry.py``),
its own separable dense-box Hamiltonian (``hamiltonian.py``), its own intersection
scalar products (``matrices.py``) and an explicit-matrix brute force for tiny boxes
(``brute.py``).  Each function cites the part of the paper it follows; where the
paper delegates a definition to the BigDFT literature, the docstring states the
reading taken.

Modules
-------
filters      Daubechies-16 least-asymmetric filter, moments, magic filter, kinetic
             connection coefficients (Sec. II.B).
geometry     grid, fine region, locregs L and L' and their segment keys, compressed
             layout, pair pattern (Sec. II.B, Sec. III, Eq. loccon, Eq. "H = L' H L").
hamiltonian  H phi = L' (T + W^T M^T V M W) L phi per support function (Sec. III.B).
matrices     S_ab = <phi_a|phi_b>, H_ab = <phi_a|H phi_b> on the CSR pattern (Sec. II.A).
brute        explicit dense matrices on tiny boxes (pin for the separable oracle).
density      rho_j = sum_ab K_ab u_a(j) u_b(j) on the fine grid (Sec. II.A, Eq. density).
confinement  quartic confining potential a (r - R)^4 in the two-level basis and the
             preconditioning equation solved by conjugate gradients (Sec. "Support
             function optimization", Eq. precond).
combine      sparse combinations P_L sum_beta M_ab phi_beta and the first-order Taylor
             Loewdin step (Sec. "Orthogonalization", Eq. gradient).
gradient     support-function gradient of the band-structure energy (Eq. gradient).
foe          density kernel by the Fermi operator expansion (App. "Fermi operator
             expansion"): Chebyshev recursion, erf smearing, bisection on mu.
"""
