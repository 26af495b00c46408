"""FP64 CPU oracle for the parabolic-operator hot path -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import this
package.  The product library (`paper_2403_01004_gb300`) never imports, links or runs it, and it
shares no code with the CUDA path: the two meet only at the seeded input generator `synth`.

Everything here is plain NumPy in float64, written to be checked against the paper by eye:

* `geometry`  - nonuniform spherical shell grid, cell volumes, corner metric factors.
* `tc`        - field-aligned thermal conduction F_tc (Eq. 2, right), lagged kappa = T0^{5/2}.
* `visc`      - artificial viscosity F_visc (Eq. 2, left) on the three staggered velocity grids.
* `sts`       - RKL2 (Sec. 3.1, the method of Meyer, Balsara & Aslam) and RKG2 (Appendix A)
                coefficients, stage counts and the s-stage recurrence.
* `ptl`       - the practical time-step limit (Eqs. 3-5) at the location of max |F|.
* `advance`   - the dynamic PTL cycle loop (Sec. 2, last paragraph) around STS or BE + PCG.
* `pcg`       - Backward Euler solved by point-Jacobi preconditioned CG (Sec. 3.1).
* `dense`     - tiny-grid dense matrices, eigen-decompositions and direct solves used as truth.

Parity unpinned: the PTL cycle schedule on the spherical workloads (no independent truth beyond
this code; the paper prints no cycle counts) -- it is pinned only through the eigenmode case,
where the schedule has a closed form.
"""
