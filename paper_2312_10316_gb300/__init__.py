"""GB300 (sm_103a) TRT-R lattice Boltzmann step for the convection-diffusion equation with
variable coefficients (arXiv 2312.10316).

``trtr`` is the Python binding of the C ABI in ``include/trtr.h`` (``libtrtr.so``);
``workloads`` generates the seeded synthetic pulse inputs; ``build`` compiles the library.
"""
__all__ = ["trtr", "workloads", "build"]
