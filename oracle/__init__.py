"""Plain FP64 CPU oracle for the MOT-JVIE march of arXiv 2407.03323.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) may import, call, link or execute anything in this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA path; the
only module both sides import is ``workloads`` (seeded inputs, no arithmetic of the
method).

Contents (each function cites the passage of the paper it follows):

* ``spline``        quadratic temporal B-spline T and T'' (Sec. 2.3, reading R1)
* ``kernel_table``  interaction-element quadrature K^vol, K^face, G (Eq. Z with S of
                    Eq. TDJVIE), cylindrical tanh-sinh route
* ``static``        static (lag-summed) element integrals by an independent
                    Cartesian tensor-Gauss/Duffy route; used only to pin the table
* ``brute``         every lag and component of the elements by a Cartesian iterated
                    rule that resolves the shells r = integer; used only to pin the table
* ``excitation``    tested incident field (Eq. E) for the modulated Gaussian plane wave
* ``march``         direct space-time sum (Eq. PnMOT) + dense Z_0 solve (Eq. MOTInversion);
                    sparse-source history from per-offset elements
* ``direct``        the same march with the history summed by plain C loops over voxel
                    pairs and lags (``direct_sum.c``) for grids whose dense Z_l do not fit
* ``pdsa``          PDSA matrices D_n (Eq. Dn), the FIR regularisation identity, and the
                    spectrum bracket of D_n from its circulant embedding (App. A; numpy
                    FFT of the embedded kernel, 3x3 eigenvalues per bin)
* ``response``      tapered frequency response |H^alpha| (Eq. Halpha) and the incident
                    pulse's amplitude spectrum
* ``probes``        scattered field at probe voxels outside the grid (objective of the
                    adjoint workload) and its transposed operator (the adjoint source)

Parity status: every function is pinned by a ``-m "not gpu"`` test against closed
forms, sum rules, exact identities or brute force, except the absolute physical
accuracy of the element values against the paper's own (semi-analytic) values, which
the paper does not print: that comparison is "parity unpinned".
"""
