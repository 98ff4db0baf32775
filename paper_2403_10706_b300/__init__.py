"""B300-native (sm_103a) hot path of PyHySCO's reversed-gradient-polarity field-map estimation
(arXiv 2403.10706): objective, gradient, Gauss-Newton Hessian-vector products, Jacobi and
per-column preconditioners, 1D optimal-transport initialisation and the GN-PCG solve, all in
hand-written CUDA behind the C ABI of include/hysco.h.

`Hysco` (torch binding) is imported lazily so that the C-ABI declarations in `_lib` and the
input generator in `phantom` stay usable without a CUDA device.
"""


def __getattr__(name):
    if name == "Hysco":
        from .hysco import Hysco
        return Hysco
    raise AttributeError(name)
