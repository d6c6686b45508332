"""FP64 CPU oracle for the Yee + embedded-ROM time-marching scheme of
Zhang, Bekmambetova and Triverio, "A Stable FDTD Method with Embedded
Reduced-Order Models" (arXiv:1609.07114).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library.

Every function is written in plain numpy/scipy, in FP64, in the order and
notation of the paper, so that it can be checked against the paper by eye:

* ``yee``        coarse 2D TEz Yee scheme (Sec. II-A, Eqs. (1), (3), (5))
* ``fine``       fine-region descriptor system (Sec. II, Eqs. (3)-(8))
* ``sprim``      structure-preserving block-Krylov projection (Sec. III)
* ``passivity``  passivity checks and CFL extension (Sec. V, Eqs. (24)-(27))
* ``couple``     coupling of a ROM to the coarse grid (Sec. IV, Eqs. (13)-(23))
* ``subgrid``    direct full-fine subgridding stepper (V = I), an independent
                 path used to pin ``couple``
* ``scheme``     the complete time loop with sources and probes (Sec. IV-C)
                 and the discrete storage function (Sec. V, Appendix A)
* ``problem``    builds a whole problem (grid + reduced models) from a
                 workload record
* ``adjoint``    exact transpose of the time loop (gradients of the probe
                 energy with respect to cell materials and source samples)

Readings of places where the paper is silent or garbled are listed in each
module header.  Parity unpinned: the accuracy of a reduced model relative to
the true fine mesh (the paper prints it only as figures).
"""
