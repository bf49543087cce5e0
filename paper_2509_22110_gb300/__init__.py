"""GB300 (sm_103a) tangent-point energy of closed triangle meshes.

Phi(X) = c * sum over ordered pairs (T, S) of triangles sharing no vertex of
w_T w_S |<nu_T, x_T - x_S>|^q / |x_T - x_S|^p  (Eq. TP, Sec. 2.2.2 of
Porrmann, Bartels, Voigt, "Self-avoiding fluid deformable surfaces"), with its
exact vertex gradient, evaluated by hand-written CUDA kernels behind the C ABI
of ``include/tp.h``.

``_tp`` is the ctypes binding (same names as the C entry points);
:class:`TPEnergy` is the ``torch.autograd.Function``: when the positions
require a gradient its forward makes one ``tp_gradient`` call (energy and
vertex gradient from a single pass over the pairs, which recomputes the pair
geometry; nothing per pair is stored) and keeps the [nv, 3] gradient for the
backward, which only scales it; otherwise the forward calls ``tp_energy``.
:class:`TangentPointEnergy` owns a context for one mesh topology.
``meshgen`` builds the seeded synthetic meshes.
"""

from __future__ import annotations

from . import _tp
from ._tp import (  # noqa: F401
    TP_BH,
    TP_BH_DUAL,
    TP_DIRECT,
    TP_F32_F64ACC,
    TP_F64,
    TP_LEARNED,
    TP_LEARNED_ENERGY,
    TPError,
    tp_conf_gradient,
    tp_conf_upload,
    tp_create,
    tp_debug_accum,
    tp_debug_tree,
    tp_debug_tri_data,
    tp_destroy,
    tp_energy,
    tp_far_model_load,
    tp_fields,
    tp_get_stats,
    tp_gradient,
    tp_last_error,
    tp_mesh_upload,
    tp_params_default,
    tp_set_learned_window,
    tp_set_quadrature,
    tp_tree_build,
    tp_version,
)

__all__ = [
    "TPEnergy",
    "tp_conf_upload",
    "tp_conf_gradient",
    "TangentPointEnergy",
    "tp_create",
    "tp_destroy",
    "tp_mesh_upload",
    "tp_tree_build",
    "tp_energy",
    "tp_gradient",
    "tp_far_model_load",
    "tp_fields",
    "tp_get_stats",
    "tp_params_default",
    "tp_set_quadrature",
]


def _torch():
    import torch

    return torch


class TangentPointEnergy:
    """A library context bound to one mesh topology on one CUDA device.

    ``params`` keyword arguments set the ``tp_params`` fields (q, p, scale,
    mode, theta, prec, flags).  Positions are re-uploaded on every call; the
    faces only when they change.
    """

    def __init__(self, F, device=0, stream=None, **params):
        torch = _torch()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx = tp_create(self.device.index or 0, stream)
        self.F = torch.as_tensor(F, dtype=torch.int32).to(self.device).contiguous()
        self.params = tp_params_default(**params)
        self._uploaded = False
        self._tree = None
        self.calls = {"energy": 0, "gradient": 0}  # library evaluations made through this object

    def close(self):
        if self.ctx:
            tp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def upload(self, V):
        V = V.detach().contiguous()
        if not self._uploaded:
            tp_mesh_upload(self.ctx, V, self.F)
            self._uploaded = True
        else:
            tp_mesh_upload(self.ctx, V, None, flags=_tp.TP_POSITIONS_ONLY)
        if self.params.mode != TP_DIRECT:
            tp_tree_build(self.ctx, 16, 30)

    def energy(self, V):
        self.upload(V)
        self.calls["energy"] += 1
        return tp_energy(self.ctx, self.params)

    def gradient(self, V, out=None):
        self.upload(V)
        torch = _torch()
        g = out if out is not None else torch.empty_like(V)
        self.calls["gradient"] += 1
        e = tp_gradient(self.ctx, g, self.params)
        return e, g

    def __call__(self, V):
        return TPEnergy.apply(V, self)


def _make_function():
    torch = _torch()

    class _TPEnergy(torch.autograd.Function):
        """Phi(V) with backward dPhi/dV from the hand-written adjoint kernel."""

        @staticmethod
        def forward(ctx, V, tpe):
            if ctx.needs_input_grad[0]:
                # one pass over the pairs gives both; only the vertex gradient is kept
                e, grad = tpe.gradient(V.detach())
                ctx.save_for_backward(grad)
            else:
                e = tpe.energy(V)
            return V.new_tensor(e)

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return grad * g, None

    return _TPEnergy


class _LazyFunction:
    _fn = None

    def __getattr__(self, name):
        if _LazyFunction._fn is None:
            _LazyFunction._fn = _make_function()
        return getattr(_LazyFunction._fn, name)


TPEnergy = _LazyFunction()
