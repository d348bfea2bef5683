"""An object interface over the C ABI of include/kg.h: argument marshalling and bookkeeping
only, every step runs in the CUDA library.  The library holds one context per process,
so one Solver is live at a time (creating another replaces the first).

    with Solver(u0, L=32.0, dt=0.005, precision="df64", energy_every=10) as s:
        s.step(200)
        E = s.energy()
        u = s.field()              # numpy, or s.field(device=True) for a torch tensor

u0 (and v0) may be numpy arrays or CUDA torch tensors, real or complex (a complex u0
selects the complex-field path, |u|^2 u on the full spectrum).
"""
import numpy as np

from . import kg


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _is_complex(a):
    if hasattr(a, "is_complex"):
        return bool(a.is_complex())
    return np.iscomplexobj(a)


class Solver:
    """Eq. (2) stepped on the GPU from (u0, v0) on an N^3 grid of side L (N = u0.shape[0])."""

    def __init__(self, u0, L, dt, v0=None, precision="df64", energy_every=0, nonlinearity=1.0,
                 blowup_threshold=0.0, drift_tol=0.0, stream=None, scheme="eq2"):
        shape = tuple(u0.shape)
        if len(shape) != 3 or len(set(shape)) != 1:
            raise ValueError("u0 must be an N x N x N array")
        self.N, self.L, self.dt = shape[0], float(L), float(dt)
        self.complex = _is_complex(u0) or (v0 is not None and _is_complex(v0))
        if stream is not None:
            kg.kg_set_stream(stream)
        kg.kg_set_options(precision=precision, energy_every=energy_every, nonlinearity=nonlinearity,
                          blowup_threshold=blowup_threshold, drift_tol=drift_tol)
        kg.kg_set_scheme(scheme)   # "eq2" (Eq. (2)) or "composed4" (fourth order, real fields)
        if _is_torch_cuda(u0):
            import torch
            u = u0.to(dtype=torch.complex128 if self.complex else torch.float64).contiguous()
            v = None if v0 is None else v0.to(device=u.device, dtype=u.dtype).contiguous()
            init = kg.kg_init_complex_device if self.complex else kg.kg_init_device
            init(self.N, self.L, self.dt, u, v)
        else:
            init = kg.kg_init_complex if self.complex else kg.kg_init
            init(self.N, self.L, self.dt, u0, v0)
        self._open = True

    # ---- stepping and diagnostics ----
    def step(self, n=1):
        """enqueue n steps (asynchronous on the library's stream); returns self"""
        kg.kg_step(int(n))
        return self

    def energy(self, allow_drift=False):
        """E^{n-1/2} at the current level (synchronises)"""
        return kg.kg_energy(allow_drift=allow_drift)

    def status(self):
        """level, frozen (blown up), blowup_level, maxabs (synchronises)"""
        return kg.kg_status()

    @property
    def level(self):
        return self.status()["level"]

    # ---- read-out ----
    def field(self, device=False):
        """u^n: a numpy array, or with device=True a CUDA torch tensor (float64, or
        complex128 for a complex field)"""
        if device:
            import torch
            dtype = torch.complex128 if self.complex else torch.float64
            out = torch.empty((self.N,) * 3, dtype=dtype, device="cuda")
            if self.complex:
                kg.kg_fetch_complex_device(out)
            else:
                kg.kg_fetch_device(out)
            return out
        return kg.kg_fetch_complex(self.N) if self.complex else kg.kg_fetch(self.N)

    def spectral(self):
        """(uh^n, uh^{n-1}) as numpy complex128 arrays"""
        return kg.kg_fetch_spectral(self.N)

    # ---- checkpoints ----
    def save(self):
        """the run as one checkpoint buffer (numpy uint8)"""
        return kg.kg_save_state()

    @classmethod
    def load(cls, buf):
        """a Solver resumed from a checkpoint buffer written by save()"""
        b = buf if isinstance(buf, np.ndarray) else np.frombuffer(buf, dtype=np.uint8)
        h = kg.state_header(b)
        kg.kg_load_state(b)   # also restores the checkpoint's scheme
        s = cls.__new__(cls)
        s.N, s.L, s.dt = h.N, h.L, h.dt
        s.complex = bool(h.complex_field)
        s._open = True
        return s

    # ---- lifetime ----
    def close(self):
        if getattr(self, "_open", False):
            kg.kg_finalize()
            self._open = False

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False
