"""torch.autograd over the C-ABI operators: E, E^H, E^H E and the CG solve, differentiable
with respect to their vector input and to the B0 map omega (row 0 of R, rad/s).

Every forward and backward step runs in the library's kernels; this module only keeps the
plan's B0 map equal to the omega tensor it is given and allocates outputs. Gradients follow
PyTorch's convention for complex tensors (dL/dRe + i dL/dIm of a real loss):

  y = E m      ->  dL/dm = E^H g,              dL/domega = Im(conj(m) E^H(t o g))
  x = E^H y    ->  dL/dy = E h,                dL/domega = Im(conj(h) E^H(t o y))
  x = CG(s)    ->  reverse mode through the unrolled iterations, replayed from checkpoints
                   taken every ckpt_every iterations (sense_cg_backward)

with t the sample times (column 0 of K). The paper only solves; the gradients serve joint
B0-map refinement and training through the reconstruction.
"""
import numpy as np
import torch

from . import native


class SenseOperator:
    """The encoding operator of one problem (a plan) in one precision mode.

    omega arguments are float32 CUDA tensors [L] in user voxel order, or None to keep the
    plan's current B0 map. A new omega rebuilds the plan's phase anchors (host work, a few
    milliseconds at 256x256); an unchanged one costs one comparison.
    """

    def __init__(self, Kmat, Rmat, S, j=None, prec="fp32"):
        self.plan = native.Plan(Kmat, Rmat, S, j)
        self.prec = native.PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.L, self.K, self.C = self.plan.L, self.plan.K, self.plan.C
        self._omega = torch.from_numpy(np.ascontiguousarray(Rmat[0], np.float64))

    def close(self):
        self.plan.close()

    def _use(self, omega):
        if omega is None:
            return
        w = omega.detach().to(torch.float64).cpu()
        if w.shape != (self.L,):
            raise ValueError(f"omega must have shape ({self.L},)")
        if not torch.equal(w, self._omega):
            native.sense_plan_set_b0(self.plan.handle, w.numpy())
            self._omega = w.clone()

    def E(self, m, omega=None):
        return _Encode.apply(m, omega, self)

    def EH(self, y, omega=None):
        return _Adjoint.apply(y, omega, self)

    def normal(self, m, omega=None):
        return self.EH(self.E(m, omega), omega)

    def cg(self, s, omega=None, n_iter=40, ckpt_every=8, rel_tol=0.0, apply_j=True):
        return _CG.apply(s, omega, self, int(n_iter), int(ckpt_every), float(rel_tol),
                         bool(apply_j))


def _c64(t):
    return t.detach().contiguous().to(torch.complex64)


def _sync(op):
    native.sense_plan_sync(op.plan.handle)


class _Encode(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, omega, op):
        op._use(omega)
        m = _c64(m)
        s = torch.empty((op.K, op.C), dtype=torch.complex64, device=m.device)
        native.sense_encode(op.plan.handle, op.prec, m, s)
        _sync(op)
        ctx.op = op
        ctx.save_for_backward(m, omega)
        return s

    @staticmethod
    def backward(ctx, g):
        m, omega = ctx.saved_tensors
        op = ctx.op
        op._use(omega)
        g = _c64(g)
        need_m, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gm = torch.empty_like(m) if need_m else None
        gw = None
        if need_w:
            gw = torch.empty(op.L, dtype=torch.float32, device=m.device)
            native.sense_grad_b0(op.plan.handle, op.prec, m, g, gw, z=gm)
        elif need_m:
            native.sense_adjoint(op.plan.handle, op.prec, g, gm)
        _sync(op)
        return gm, gw, None


class _Adjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, omega, op):
        op._use(omega)
        y = _c64(y)
        x = torch.empty(op.L, dtype=torch.complex64, device=y.device)
        native.sense_adjoint(op.plan.handle, op.prec, y, x)
        _sync(op)
        ctx.op = op
        ctx.save_for_backward(y, omega)
        return x

    @staticmethod
    def backward(ctx, h):
        y, omega = ctx.saved_tensors
        op = ctx.op
        op._use(omega)
        h = _c64(h)
        gy = gw = None
        if ctx.needs_input_grad[0]:
            gy = torch.empty_like(y)
            native.sense_encode(op.plan.handle, op.prec, h, gy)
        if ctx.needs_input_grad[1]:
            gw = torch.empty(op.L, dtype=torch.float32, device=y.device)
            native.sense_grad_b0(op.plan.handle, op.prec, h, y, gw)
        _sync(op)
        return gy, gw, None


class _CG(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s, omega, op, n_iter, ckpt_every, rel_tol, apply_j):
        op._use(omega)
        s = _c64(s)
        nbytes = native.sense_cg_ckpt_bytes(op.plan.handle, n_iter, ckpt_every)
        ck = torch.empty(nbytes, dtype=torch.uint8, device=s.device)
        x = torch.empty(op.L, dtype=torch.complex64, device=s.device)
        info = native.sense_cg_solve_ckpt(op.plan.handle, s, x, ck, n_iter, ckpt_every,
                                          prec=op.prec, rel_tol=rel_tol, apply_j=apply_j)
        _sync(op)
        ctx.op = op
        ctx.info = info
        ctx.save_for_backward(s, omega, ck)
        return x

    @staticmethod
    def backward(ctx, xbar):
        s, omega, ck = ctx.saved_tensors
        op = ctx.op
        op._use(omega)
        need_s, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_s or need_w):
            return (None,) * 7
        sbar = torch.empty_like(s) if need_s else None
        wbar = torch.empty(op.L, dtype=torch.float32, device=s.device) if need_w else None
        native.sense_cg_backward(op.plan.handle, s, ck, _c64(xbar), sbar=sbar, omega_bar=wbar)
        _sync(op)
        return sbar, wbar, None, None, None, None, None
