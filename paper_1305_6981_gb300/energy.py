"""Energy functional E(h, V; c) = c^T H c / c^T c of a fixed amplitude vector, differentiable in the
integrals: the forward pass and the backward pass (the 1- and 2-RDMs of c) run in libfciqmc.so
(include/fciqmc.h, fciqmc_rdm_*); this module only marshals arguments."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import check


class EnergyFunctional:
    """Connected-pair structure of a fixed list of determinants with amplitudes c, on one GPU.

    dets: (n, W) uint64 (numpy or torch), distinct; c: (n,) float64. The integrals are passed per call.
    """

    def __init__(self, n_elec: int, n_orb: int, dets, c, device=None, stream=None):
        import torch

        self._L = L = _native.load()
        self.n_elec, self.n_orb = int(n_elec), int(n_orb)
        self.W = (2 * n_orb + 63) // 64
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        d = torch.as_tensor(np.ascontiguousarray(np.asarray(dets, dtype=np.uint64).reshape(-1, self.W)).view(np.int64)
                            if not isinstance(dets, torch.Tensor) else dets).to(dev).contiguous()
        cc = torch.as_tensor(c, dtype=torch.float64).to(dev).contiguous()
        self.n = int(cc.numel())
        nbytes = L.fciqmc_rdm_workspace_bytes(self.n_elec, self.n_orb, self.n)
        if nbytes == 0:
            raise ValueError("unsupported problem size")
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            rc = L.fciqmc_rdm_create(self.n_elec, self.n_orb, ctypes.c_void_p(d.data_ptr()),
                                     ctypes.c_void_p(cc.data_ptr()), self.n, ctypes.c_void_p(self.workspace.data_ptr()),
                                     int(nbytes), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        check(rc, "fciqmc_rdm_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self._L.fciqmc_rdm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def energy(self, h, eri):
        """E for device float64 tensors h (n_orb, n_orb) and eri (packed); returns a 0-dim device tensor."""
        import torch
        h = h.contiguous()
        eri = eri.contiguous()
        e = torch.empty((), dtype=torch.float64, device=self.device)
        check(self._L.fciqmc_rdm_energy(self.handle, ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(eri.data_ptr()),
                                        ctypes.c_void_p(e.data_ptr())), "fciqmc_rdm_energy")
        return e

    def gradient(self, scale):
        """(scale dE/dh, scale dE/dV) for a 0-dim device float64 tensor scale."""
        import torch
        npair = self.n_orb * (self.n_orb + 1) // 2
        gh = torch.empty((self.n_orb, self.n_orb), dtype=torch.float64, device=self.device)
        ge = torch.empty(npair * (npair + 1) // 2, dtype=torch.float64, device=self.device)
        s = scale.to(torch.float64).contiguous()
        check(self._L.fciqmc_rdm_gradient(self.handle, ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(gh.data_ptr()),
                                          ctypes.c_void_p(ge.data_ptr())), "fciqmc_rdm_gradient")
        return gh, ge

    def info(self) -> dict:
        out = (ctypes.c_int64 * 5)()
        check(self._L.fciqmc_rdm_info(self.handle, out), "fciqmc_rdm_info")
        return dict(zip(["buckets", "members", "candidate_pairs", "single_pairs", "double_pairs"], list(out)))


def _autograd_function():
    import torch

    class RdmEnergy(torch.autograd.Function):
        """E(h, V; c) with dE/dh and dE/dV from the density matrices (hand-written backward kernels)."""

        @staticmethod
        def forward(ctx, h, eri, functional):
            ctx.functional = functional
            return functional.energy(h.detach(), eri.detach())

        @staticmethod
        def backward(ctx, grad_out):
            gh, ge = ctx.functional.gradient(grad_out.detach())
            return gh, ge, None

    return RdmEnergy


_RDM = None


def rdm_energy(h, eri, functional: EnergyFunctional):
    """Differentiable E(h, V; c) (a torch.autograd.Function)."""
    global _RDM
    if _RDM is None:
        _RDM = _autograd_function()
    return _RDM.apply(h, eri, functional)
