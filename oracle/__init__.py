"""CPU oracle for the Parareal advection-diffusion path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA path.

Modules
-------
``oracle.core``     ctypes wrappers around the plain C FP64 routines of
                    ``oracle.c`` (stencils, RK4, Euler, restriction,
                    prolongation, shift, 3-D convolution, GELU).
``oracle.parareal`` serial Parareal exactly as Eq. (parareal) / Algorithm 1,
                    with the propagators built from ``oracle.core``.
``oracle.modal``    exact discrete solution per Fourier mode (numpy), the
                    analytic solution of Sec. 3 and the speedup model of
                    Sec. 2.2.2.
``oracle.spectral`` Fourier restriction and prolongation between the fine
                    and the coarse grid (numpy FFT), Sec. 2.2.2.
``oracle.net``      forward / backward of the learned coarse propagator's
                    convolution net, plain FP64, and one Adam step.
"""
