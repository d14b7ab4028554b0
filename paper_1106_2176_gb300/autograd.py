"""Differentiable weighted energy of the FMM potential.

E(x, q, w) = 1/2 sum_i w_i q_i phi_i, phi_i = sum_{j != i} q_j / |x_i - x_j|,
evaluated by the FMM. The backward pass is the library's adjoint: the kernel
is symmetric, so dE/dq and dE/dx need one more FMM evaluation on the same tree
with charges w q (psi), and nothing of the forward pass is kept but phi and
grad phi; the expansions are recomputed rather than stored.

    E = fmm_energy(x, q, w, p=8, theta=0.5, ncrit=64, precision="mixed")
    E.backward()   # x.grad, q.grad, w.grad
"""
import threading
import weakref

import torch

from .fmm import FMM

# Handles (and their device workspaces) are reused across calls with the same
# size and parameters: a forward pass leases one, and the lease goes back to
# the pool after the backward pass, or when the autograd graph is freed
# without a backward pass.
_pool = {}
_pool_lock = threading.Lock()
POOL_MAX = 4  # idle handles kept per key


def _take(n, p, theta, ncrit, precision, device):
    key = (int(n), int(p), float(theta), int(ncrit), precision, device)
    with _pool_lock:
        free = _pool.get(key)
        if free:
            return key, free.pop()
    return key, FMM(n, p=p, theta=theta, ncrit=ncrit, precision=precision)


def _give(key, f):
    with _pool_lock:
        free = _pool.setdefault(key, [])
        if len(free) < POOL_MAX:
            free.append(f)
            return
    f.close()


def clear_pool():
    """Close every idle pooled handle."""
    with _pool_lock:
        hs = [f for free in _pool.values() for f in free]
        _pool.clear()
    for f in hs:
        f.close()


class _Lease:
    """A pooled handle held by one forward pass; returned exactly once, by
    release() or, failing that, when the lease is garbage collected."""

    def __init__(self, key, f):
        self.f = f
        self._fin = weakref.finalize(self, _give, key, f)

    def release(self):
        self.f = None
        self._fin()


class FMMEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, q, w, p, theta, ncrit, precision):
        key, f = _take(x.shape[0], p, theta, ncrit, precision, str(x.device))
        ctx.lease = _Lease(key, f)
        ctx.args = (p, theta, ncrit, precision)
        x, q, w = x.contiguous(), q.contiguous(), w.contiguous()
        f.build(x, q)
        phi, grad = f.evaluate()
        e = f.energy(w, q, phi)
        ctx.save_for_backward(x, q, w, phi, grad)
        return torch.tensor(e, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, gE):
        x, q, w, phi, grad = ctx.saved_tensors
        lease = ctx.lease
        if lease.f is None:
            # a second backward (retain_graph=True): the first one returned
            # the handle, so lease another and rebuild the tree of x
            p, theta, ncrit, precision = ctx.args
            lease = _Lease(*_take(x.shape[0], p, theta, ncrit, precision, str(x.device)))
            lease.f.build(x, q)
        f = lease.f
        f.update_charges(q, w)
        psi, gpsi = f.evaluate()
        dq, dx, dw = f.energy_adjoint(float(gE), w, q, phi, grad, psi, gpsi, dq=ctx.needs_input_grad[1],
                                      dx=ctx.needs_input_grad[0], dw=ctx.needs_input_grad[2])
        lease.release()
        return dx, dq, dw, None, None, None, None


def fmm_energy(x, q, w, p=8, theta=0.5, ncrit=64, precision="mixed"):
    """1/2 sum w q phi with gradients for x (n, 3), q (n,) and w (n,); CUDA tensors, float32 or float64."""
    return FMMEnergy.apply(x, q, w, p, theta, ncrit, precision)
