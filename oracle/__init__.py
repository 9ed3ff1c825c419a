"""Oracle: a plain, slow, FP64 CPU restatement of the Fourier-accelerated volume
integral method (Frerot, Bonnet, Molinari & Anciaux, arXiv:1811.11558).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_1811_11558_gb300``) never imports, calls or links it,
and it never imports the product path: the two share no code.

Modules
-------
tensors     symmetric-tensor storage, Hooke's law, deviator (Sec. 1, Sec. 4.1)
kernels     Kelvin / Boussinesq-Cerruti coefficient tensors and the gradient
            recurrence in partial Fourier space (Sec. 2.2, Table 1, Eq. recurrence)
operators   discretised Mindlin and Boussinesq operators: DFT in-plane (Thm 1,
            Eq. dft), dense O(Nz^2) Gauss-Legendre depth quadrature against the
            piecewise-linear interpolant (Sec. 3.2), no cutoff
plasticity  J2 return map with linear isotropic hardening (Sec. 4.1), DF-SANE
            (Sec. 4.3, La Cruz, Martinez & Raydan 2006)
contact     Polonsky-Keer constrained conjugate gradient (Sec. 5.1) and the
            elastic-plastic coupling of Algorithm 1 (Sec. 5.2)

Parity status of each function is stated in its module header.
"""
