"""FP64 CPU oracle for the spatial Bayesian fMRI GLM sampler (Siden, Eklund, Bolin & Villani,
"Fast Bayesian whole-brain fMRI analysis with spatial 3D priors").

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or execute this
package: only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it. It shares no code with the CUDA library
(no kernels, headers, helpers, tables or pre/post-processing); the only common input is
the seeded synthetic workload generator, which holds none of the method's arithmetic.

Everything is plain numpy / scipy in float64, written for a reader to check against the
paper by eye: the posterior precision is assembled as an explicit sparse matrix in the
paper's own ordering w_r = vec(W') (regressor-major), solves are exact (sparse LU /
dense Cholesky), and each function cites the passage it follows.

Modules
-------
lattice  -- in-mask voxel graph: compact indexing, edge list (G_w), D_w (Section 2; Eq. 6)
philox   -- Philox4x32-10 counter-based generator, Box-Muller normals, Rademacher signs,
            Marsaglia-Tsang Gamma draws (published definitions; the paper is silent)
model    -- whitening, sufficient statistics, full conditionals of W, A, lambda, alpha,
            beta (Appendix A, temporal noise model), perturbed right-hand side (Algorithm 2)
linalg   -- exact sparse solves, log-determinants, Lanczos / stochastic Lanczos quadrature
gibbs    -- one Gibbs sweep (Section 3.2) and one spatial-VB step (Section 3.3, Appendix B/C)
probes   -- exact log-determinant and trace terms behind the stochastic probes
precond  -- block-Jacobi and red-black symmetric SOR preconditioners (replacing the
            incomplete Cholesky of Section 3.1), factored form and voxel-by-voxel sweeps
multigrid -- aggregation multigrid V-cycle (Galerkin coarse operators, symmetric red-black
            block Gauss-Seidel smoothing) as a further replacement
summaries -- posterior summaries: chain PPMs and joint PPMs (Eq. MCMCPPM, Eq. MCMCjointPPM),
            SVB sample moments and Gaussian PPMs (Section 3.3), the unnormalised log joint
            posterior (Eq. UnnormalisedJointPosterior)

Parity status: every function is pinned by a ``-m "not gpu"`` test against a closed form,
an invariant, an independent library routine or brute force. The SVB extrapolation of
Appendix C (``gibbs.svb_extrapolate``), for which the paper prints no iterate values, is
pinned branch by branch to values worked by hand from the rule the appendix states; its
fallback for a non-positive prediction is a reading, not the paper's.
"""
