"""Helpers shared by the GPU parity tests (inputs from odwf_synth, references from oracle/)."""
import numpy as np
import pytest

import odwf_synth as syn
from oracle import zolotarev

M0 = 1.3


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def assert_close_componentwise(got, ref, tol):
    """|got - ref| <= tol * max(|ref|, 1e-3 ||ref||_inf) elementwise (near-zero components are
    judged against the field's scale)."""
    got = np.asarray(got).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    err = np.abs(got - ref) / scale
    assert err.max() <= tol, "max scaled error %.3e > %.1e" % (err.max(), tol)
    return err.max()


def rel_norm(a, b):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)).reshape(-1)) / np.linalg.norm(np.asarray(b).reshape(-1))


def make_case(dims, ns, mq, eps=0.3, seed=1, lrange=(0.05, 6.0), shifted=True):
    U = syn.gauge_field(dims, eps, seed)
    w, _ = zolotarev.omega(ns, lrange[0], lrange[1], shifted)
    return U, w


def to_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def from_dev(t):
    return t.cpu().numpy()
