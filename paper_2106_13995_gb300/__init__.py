"""GB300-native Schroedinger state-vector simulator.

The state (2^n complex amplitudes) stays in GPU memory and gates are applied
to it in place by hand-written sm_103a CUDA kernels behind a C ABI
(``include/sv_api.h``, library ``_build/libsv.so``).  This package holds the
build script, a thin ctypes binding (``sim``), a circuit builder with Pauli
observables and a simulator facade (``circuit``), and the multi-GPU sharding
planner and executor (``shard``).
"""
from . import _native  # noqa: F401
from .circuit import Circuit, I, Parameter, PauliSum, Simulator, X, Y, Z, grid_qubit, ising  # noqa: F401


def build(force: bool = False) -> str:
    from .buildlib import build as _b
    return _b(force=force)


def __getattr__(name):
    # lazy import so that `import paper_2106_13995_gb300` works without torch/CUDA
    if name in ("StateVector", "adjoint_grad", "adjoint_grad_batch", "marshal", "options",
                "SvExpectation", "kernel_launches", "pauli_terms", "sim"):
        import importlib
        sim = importlib.import_module(__name__ + ".sim")
        return sim if name == "sim" else getattr(sim, name)
    raise AttributeError(name)
