"""torch.autograd.Function for C = A B with the hand-written backward of libshiro.

Forward: pack B's rows named by every tile's Cols and SpMM over the packed rows (one library
call, shiro_pack_spmm).  Backward: dB = A^T dC through the TRANSPOSE plan (pack dC, SpMM) and
dA = SDDMM(dC, B) on A's pattern, in one library call (shiro_spmm_backward); for rows of 256 or
512 bytes both come from one launch that gathers each dC row once.  All of it runs in the CUDA
library.
"""
from __future__ import annotations

import torch

from . import shiro


class SparseMatrix:
    """CSR A on the GPU with its forward plan and the plan of A^T (built once per pattern)."""

    def __init__(self, rowptr, col, val, M, K, P_r=1, P_c=1, flags=0, opts=None,
                 transpose=True):
        self.rowptr, self.col, self.M, self.K = rowptr, col, M, K
        self.val = val
        self.plan = shiro.Plan.create(rowptr, col, val, M, K, P_r, P_c, flags=flags, opts=opts)
        self.planT = None
        if transpose:
            self.planT = shiro.Plan.create(rowptr, col, val, M, K, P_r, P_c,
                                           flags=flags | shiro.SHIRO_PLAN_TRANSPOSE, opts=opts)
        self._val_version = val._version

    def sync_values(self, val):
        """Reload A^T's values when A's value tensor changed since the last call."""
        if self.planT is not None and (val is not self.val or val._version != self._val_version):
            self.planT.update_values(val)
            self.val = val
            self._val_version = val._version


class ShiroSpMM(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A: SparseMatrix, val, B):
        if val is not A.val:
            raise ValueError("val must be the value tensor the plan was built on")
        Bc = B.contiguous()
        Bpack = torch.empty((A.plan.info.packed_rows, Bc.shape[1]), dtype=Bc.dtype,
                            device=Bc.device)
        C = A.plan.pack_spmm(Bc, Bpack=Bpack)
        ctx.A = A
        ctx.save_for_backward(Bpack, Bc)
        return C

    @staticmethod
    def backward(ctx, dC):
        A = ctx.A
        Bpack, Bc = ctx.saved_tensors
        want_dA = ctx.needs_input_grad[1]
        want_dB = ctx.needs_input_grad[2]
        dC = dC.contiguous().to(Bc.dtype)
        if want_dB:
            A.sync_values(A.val)
        dB, dA = shiro.spmm_backward(A.plan, A.planT, dC, Bpack, B=Bc, want_dB=want_dB,
                                     want_dA=want_dA)
        return None, dA, dB


def spmm(A: SparseMatrix, B):
    """C = A B with autograd support for A's values and for B."""
    return ShiroSpMM.apply(A, A.val, B)
