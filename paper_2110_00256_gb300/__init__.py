"""GB300-native strong-field QED Monte Carlo substep (PICSAR-QED, Fedeli et al.,
arXiv 2110.00256): CUDA kernels for sm_103a behind the C ABI of include/qed.h.

``paper_2110_00256_gb300.api`` is the Python binding (needs torch and the built
``_build/libqed.so``); ``paper_2110_00256_gb300.build`` compiles the library;
``paper_2110_00256_gb300.workloads`` draws the seeded synthetic inputs.
"""
__all__ = ["api", "build", "workloads"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
