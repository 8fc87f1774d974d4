"""Request server: continuous batching gives every request the result it
gets alone; bounded waits time out; admission respects the memory budget."""
import numpy as np
import pytest

import paper_2509_05047_gb300 as psc
import workloads as W

pytestmark = pytest.mark.gpu


class World:
    def __init__(self, budget=0, gaps=0):
        import torch
        from paper_2509_05047_gb300 import build
        build.build()
        self.torch = torch
        self.ctx = psc.psc_create(0, budget)
        self.sc = W.scanner_tiny()
        if gaps:  # 72 modules of 4 crystals, 4 blocks of 4 rings, 1 mm gaps
            self.sc.gap_mode, self.sc.gap_t, self.sc.gap_a = gaps, 1.0, 1.0
        self.s = psc.psc_load_scanner(self.ctx, psc.scanner_desc(self.sc))
        m = psc.psc_load_materials(self.ctx, psc.materials_desc(W.standard_materials()).desc)
        self.phantoms = [W.phantom_water_cylinder(),
                         W.phantom_random_torso(5, (40, 40, 16), voxel=(4.0, 4.0, 4.0)),
                         W.phantom_random_torso(6, (48, 48, 20), voxel=(3.0, 3.0, 3.0))]
        self.p = [psc.psc_load_phantom(self.ctx, psc.phantom_desc(ph).desc, m) for ph in self.phantoms]
        self.lut = psc.psc_load_lut(self.ctx, psc.lut_desc(W.lut_tiny(self.sc)).desc)
        self.sens = psc.psc_load_sinogram(self.ctx, self.s, W.sensitivity_uniform(self.sc.lor_shape), True)

    def out(self):
        return self.torch.full(self.sc.shape, np.nan, dtype=self.torch.float64, device="cuda")

    def alone(self, reqs):
        """Each request on its own: activity, zero, simulate, finalize."""
        stream = self.torch.cuda.current_stream().cuda_stream
        a = psc.psc_acc_create(self.ctx, self.s)
        outs = []
        for r in reqs:
            if r.get("activity") is not None:
                psc.psc_update_activity(self.ctx, self.p[r["ph"]], r["activity"])
            psc.psc_acc_zero(self.ctx, a, stream)
            psc.psc_simulate(self.ctx, psc.sim_args(r["seed"], 0, r["n"], self.s, self.p[r["ph"]], a,
                                                    lut=self.lut), stream=stream)
            o = self.out()
            psc.psc_finalize(self.ctx, psc.finalize_args(a, sens=self.sens, sigma=r.get("sigma"),
                                                         scale=1.0 / r["n"]), o, stream)
            outs.append(o)
        self.torch.cuda.synchronize()
        psc.psc_unload(self.ctx, a)
        return outs

    def served(self, reqs, **cfg):
        psc.psc_server_start(self.ctx, **cfg)
        outs = [self.out() for _ in reqs]
        # the server writes on its own streams: the fills must be complete
        self.torch.cuda.synchronize()
        tickets = []
        for r, o in zip(reqs, outs):
            tickets.append(psc.psc_submit(self.ctx, psc.request(
                self.s, self.p[r["ph"]], o, r["n"], r["seed"], lut=self.lut, sens=self.sens,
                sigma=r.get("sigma"), scale=1.0 / r["n"], activity=r.get("activity"))))
        for t in tickets:
            psc.psc_wait(self.ctx, t)
        status = [psc.psc_poll(self.ctx, t) for t in tickets]
        psc.psc_server_stop(self.ctx)
        return outs, status

    def close(self):
        psc.psc_destroy(self.ctx)


def _requests(world):
    rng = np.random.default_rng(8)
    base = world.phantoms[1].activity
    return [
        {"ph": 0, "n": 300_000, "seed": 1, "sigma": (2.0, 2.0, 2.0)},
        {"ph": 1, "n": 50_001, "seed": 2, "activity": base},
        {"ph": 2, "n": 120_000, "seed": 3},
        {"ph": 1, "n": 70_000, "seed": 4, "activity": (base * rng.uniform(0.5, 1.5, base.shape)).astype(np.float32)},
        {"ph": 0, "n": 1_000, "seed": 5, "sigma": (1.0, 1.5, 0.5)},
        {"ph": 1, "n": 90_000, "seed": 6, "activity": (base * rng.uniform(0.5, 1.5, base.shape)).astype(np.float32),
         "sigma": (2.0, 2.0, 2.0)},
        {"ph": 2, "n": 400_000, "seed": 7},
    ]


@pytest.mark.parametrize("gaps", [0, 2])
def test_served_results_equal_alone(gaps):
    """Also on a scanner with gaps (edge-crystal assignment, LUT positions of
    the virtual crystals): the batched launches carry each job's scanner."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = World(gaps=gaps)
    try:
        reqs = _requests(w)
        ref = w.alone(reqs)
        psc.psc_update_activity(w.ctx, w.p[1], w.phantoms[1].activity)
        got, status = w.served(reqs, max_active=3, epoch_histories=200_000, min_slice=4096)
        for r, a, b, st in zip(reqs, ref, got, status):
            assert st["state"] == psc.PSC_REQ_DONE
            assert st["t_submit"] <= st["t_start"] <= st["t_done"]
            assert bool((a == b).all()), f"request {r['seed']} differs in the mix"
            assert float(a.sum()) > 0
    finally:
        w.close()


def test_wait_is_bounded_and_admission_respects_budget():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    probe = World()
    resident = psc.psc_resident_bytes(probe.ctx)
    probe.close()
    acc_bytes = W.scanner_tiny().n_bins * 8
    w = World(budget=resident + acc_bytes + acc_bytes // 2)   # room for one accumulator
    try:
        reqs = [{"ph": i % 3, "n": 200_000 + 1000 * i, "seed": 20 + i} for i in range(4)]
        psc.psc_server_start(w.ctx, max_active=4, epoch_histories=100_000, min_slice=4096)
        outs = [w.out() for _ in reqs]
        torch.cuda.synchronize()
        tickets = [psc.psc_submit(w.ctx, psc.request(w.s, w.p[r["ph"]], o, r["n"], r["seed"], lut=w.lut,
                                                     sens=w.sens, scale=1.0 / r["n"]))
                   for r, o in zip(reqs, outs)]
        with pytest.raises(psc.PscError) as e:
            psc.psc_wait(w.ctx, tickets[-1], 1)
        assert e.value.code == psc.PSC_ETIMEOUT
        for t in tickets:
            psc.psc_wait(w.ctx, t)
        st = sorted((psc.psc_poll(w.ctx, t) for t in tickets), key=lambda x: x["t_start"])
        psc.psc_server_stop(w.ctx)
        # only one accumulator fits: each request starts after the previous ended
        for prev, nxt in zip(st[:-1], st[1:]):
            assert nxt["t_start"] >= prev["t_done"]
        ref = w.alone(reqs)
        for a, b in zip(ref, outs):
            assert bool((a == b).all())
    finally:
        w.close()
