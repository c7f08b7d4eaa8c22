"""Second-order Trotter-Suzuki time step of one particle on a 2-D lattice,
hand-written CUDA for sm_103a behind a C ABI (``libtrotter.so``).

``paper_1208_2407_gb300.trotter`` is the Python binding (argument marshalling
only); it loads the compiled library on first use and raises if it is absent.
``paper_1208_2407_gb300.workloads`` draws the seeded synthetic inputs.
"""

__all__ = ["trotter", "workloads"]


def __getattr__(name):
    if name in ("trotter", "workloads", "build", "autograd"):
        import importlib
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
