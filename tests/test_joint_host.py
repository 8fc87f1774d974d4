"""Host logic of the joint activity/scatter driver (Sec. 2.4.2, third
scenario), with the library calls replaced by recorders: the order of the
steps, the history range of each iteration, the finalize scale, and the
activity handed from one reconstruction to the next simulation."""
import pytest

import paper_2509_05047_gb300.joint as J


def test_iteration_order_and_history_ranges(monkeypatch):
    log = []
    monkeypatch.setattr(J, "psc_update_activity", lambda ctx, ph, a: log.append(("activity", a)))
    monkeypatch.setattr(J, "psc_acc_zero", lambda ctx, acc, s: log.append(("zero", acc)))
    monkeypatch.setattr(J, "sim_args", lambda seed, first, n, *a, **k: (seed, first, n))
    monkeypatch.setattr(J, "psc_simulate", lambda ctx, args, stream=None: log.append(("simulate", args)))
    monkeypatch.setattr(J, "finalize_args", lambda acc, **k: k)
    monkeypatch.setattr(J, "psc_finalize", lambda ctx, fin, out, s: log.append(("finalize", fin["scale"])))
    recon = []

    def reconstruct(est, i):
        recon.append((est, i))
        return f"act{i + 1}"

    last = J.scatter_iterations("ctx", 1, 2, 3, "act0", reconstruct, 3, 1000, 7, "out", first_history=50)
    assert last == "act2"
    assert recon == [("out", 0), ("out", 1)]
    steps = [e[0] for e in log]
    assert steps == ["activity", "zero", "simulate", "finalize"] * 3
    assert [e[1] for e in log if e[0] == "activity"] == ["act0", "act1", "act2"]
    assert [e[1] for e in log if e[0] == "simulate"] == [(7, 50, 1000), (7, 1050, 1000), (7, 2050, 1000)]
    assert all(e[1] == pytest.approx(1e-3) for e in log if e[0] == "finalize")


def test_rejects_empty_runs():
    with pytest.raises(ValueError):
        J.scatter_iterations("ctx", 1, 2, 3, "a", lambda e, i: e, 1, 0, 7, "out")
