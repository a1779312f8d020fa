"""Shared helpers of the GPU parity tests: torch device buffers in, numpy out."""
import numpy as np
import torch

from paper_1801_05358_gb300 import dmwf


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def alm_dev(a):
    return dev(np.ascontiguousarray(a, dtype=np.complex128).view(np.float64))


def alm_host(t, shape):
    return t.cpu().numpy().view(np.complex128).reshape(shape)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def make_plan(wl, batch=1, **sched):
    p = dmwf.Plan(wl.nside, wl.lmax, batch)
    p.set_spectra(wl.cl)
    p.set_noise_mask(wl.sigma, wl.mask)
    if sched:
        p.set_schedule(**sched)
    return p
