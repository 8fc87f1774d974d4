"""Helpers for the GPU tests: a context with loaded objects, listmode runs
through the C ABI, and the per-history comparison with the oracle."""
import numpy as np
import torch

import paper_2509_05047_gb300 as psc


class Session:
    """One psc context on cuda:0 with a scanner, materials, phantom and LUT."""

    def __init__(self, scanner, mats, phantom, lut=None, lut_dtype=psc.PSC_LUT_F32, budget=0):
        from paper_2509_05047_gb300 import build
        build.build()
        self.dev = torch.device("cuda:0")
        self.sc = scanner
        self.ctx = psc.psc_create(0, budget)
        self.s_id = psc.psc_load_scanner(self.ctx, psc.scanner_desc(scanner))
        self.m_id = psc.psc_load_materials(self.ctx, psc.materials_desc(mats).desc)
        self.p_id = psc.psc_load_phantom(self.ctx, psc.phantom_desc(phantom).desc, self.m_id)
        self.l_id = psc.psc_load_lut(self.ctx, psc.lut_desc(lut, lut_dtype).desc) if lut is not None else 0
        self.a_id = psc.psc_acc_create(self.ctx, self.s_id)

    def stream(self):
        return torch.cuda.current_stream().cuda_stream

    def run(self, seed, first, n, listmode=True, lut=None, acc=None, phantom=None, bin_mask=1,
            block=0, grid=0, stats=True):
        cls = key = q = None
        if listmode:
            cls = torch.full((max(n, 1),), -1, dtype=torch.int8, device=self.dev)
            key = torch.full((max(n, 1),), -2, dtype=torch.int64, device=self.dev)
            q = torch.full((max(n, 1),), -2, dtype=torch.int64, device=self.dev)
        args = psc.sim_args(seed, first, n, self.s_id, phantom or self.p_id,
                            self.a_id if acc is None else acc,
                            lut=self.l_id if lut is None else lut, bin_mask=bin_mask,
                            block=block, grid=grid, cls_out=cls, key_out=key, q_out=q)
        st = psc.psc_simulate(self.ctx, args, stats=stats, stream=self.stream())
        torch.cuda.synchronize()
        out = {"stats": st}
        if listmode:
            out.update(cls=cls[:n].cpu().numpy(), key=key[:n].cpu().numpy(), q=q[:n].cpu().numpy())
        return out

    def acc(self, acc=None):
        t = torch.empty(self.sc.n_bins, dtype=torch.int64, device=self.dev)
        psc.psc_acc_read(self.ctx, self.a_id if acc is None else acc, t, self.stream())
        torch.cuda.synchronize()
        return t

    def zero(self, acc=None):
        psc.psc_acc_zero(self.ctx, self.a_id if acc is None else acc, self.stream())

    def close(self):
        psc.psc_destroy(self.ctx)


def compare_histories(gpu, ref, min_match=0.999, w_rtol=1e-5):
    """>= min_match of histories in the same class and bin; fixed-point
    weight relative error <= w_rtol on those that are binned.  Returns the
    mask of matching histories."""
    same = (gpu["cls"] == ref["cls"]) & (gpu["key"] == ref["key"])
    frac = same.mean() if same.size else 1.0
    assert frac >= min_match, f"{frac:.6f} of histories match (need {min_match})"
    det = same & (ref["key"] >= 0)
    if det.any():
        rel = np.abs(gpu["q"][det] - ref["q"][det]) / ref["q"][det].astype(np.float64)
        assert rel.max() <= w_rtol, f"max weight rel err {rel.max():.3g} > {w_rtol}"
    return same


def sinogram_from(keys, qs, cls, n_bins, classes=(7,)):
    acc = np.zeros(n_bins, dtype=np.int64)
    m = np.isin(cls, classes) & (keys >= 0)
    np.add.at(acc, keys[m], qs[m])
    return acc
