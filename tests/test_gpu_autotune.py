"""The team-size autotuner: every candidate team gives the oracle's answer, the fastest is
kept per size class, forced teams (including CTAs that own no rows) stay correct, and the
JSON cache round-trips."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import phipm_oracle as O
from paper_0907_4631_gb300 import phipm as pm
from paper_0907_4631_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    pr = wl.convdiff_2d_problem(N=64, p=2, t_end=1e-3, tol=1e-8, seed=2064)
    ref, _ = O.phipm(pr.t_end, pr.op, pr.b, pr.tol, pr.symm)
    return pr, ref


def _rel(u, ref):
    return float(np.linalg.norm(u.cpu().numpy() - ref) / np.linalg.norm(ref))


def test_autotune_picks_a_measured_team(case):
    pr, ref = case
    s = pm.Phipm("f64pair")
    A = pm.DeviceOperator(pr.op)
    b = [torch.as_tensor(x).cuda() for x in pr.b]
    assert s.team_for(0, pr.n) == 1                     # default below n = 16384: one CTA
    rep = s.autotune(pr.t_end, A, b, pr.tol, pr.symm)
    teams = [t for t, _ in rep]
    assert teams[0] == 1 and len(teams) >= 4 and all(pr.n >= 64 * t for t in teams)
    best = min(rep, key=lambda e: e[1])[0]
    assert s.team_for(0, pr.n) == best
    assert s.team_for(0, 2 * pr.n) == 1                 # another size class is untouched
    u, st, _ = s.solve(pr.t_end, A, b, pr.tol, pr.symm)
    assert _rel(u, ref) <= 1e-8


@pytest.mark.parametrize("team", [1, 2, 8, 64, 152])
def test_forced_teams_match_the_oracle(case, team):
    """team 152 on n = 4096 leaves most CTAs without rows; they still join every barrier."""
    pr, ref = case
    s = pm.Phipm("f64pair")
    s.set_team(team)
    A = pm.DeviceOperator(pr.op)
    b = [torch.as_tensor(x).cuda() for x in pr.b]
    u, st, _ = s.solve(pr.t_end, A, b, pr.tol, pr.symm)
    assert _rel(u, ref) <= 1e-8


def test_tuning_cache_round_trip(case, tmp_path):
    pr, _ = case
    s = pm.Phipm("f64pair")
    A = pm.DeviceOperator(pr.op)
    b = [torch.as_tensor(x).cuda() for x in pr.b]
    s.autotune(pr.t_end, A, b, pr.tol, pr.symm)
    path = tmp_path / "tune.json"
    s.tune_save(path)
    doc = json.loads(path.read_text())
    assert doc["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert len(doc["entries"]) == 1 and doc["entries"][0]["log2n"] == 12
    s2 = pm.Phipm("f64pair")
    s2.tune_load(path)
    assert s2.team_for(0, pr.n) == s.team_for(0, pr.n)
    other = tmp_path / "other.json"
    other.write_text(json.dumps({"sms": doc["sms"] + 1, "entries": [dict(doc["entries"][0], team=3)]}))
    s3 = pm.Phipm("f64pair")
    s3.tune_load(other)                                  # another GPU's table: ignored
    assert s3.team_for(0, pr.n) == 1
    bad = tmp_path / "bad.json"
    bad.write_text('{"sms": %d, "entries": [{"precision": 2, "kind": 0}]}' % doc["sms"])
    with pytest.raises(pm.PhipmError):
        s3.tune_load(bad)
    assert s3.team_for(0, pr.n) == 1


def test_batched_autotune_picks_a_measured_cluster_size(tmp_path):
    """phipm_autotune_batched times K = 1, 2, 4, 8 CTAs per problem on the batch, keeps the
    fastest for the batch class, every K's results match the oracle, later batches of the
    class use it, and the table round-trips through the JSON cache."""
    probs = wl.batched_convdiff_problems(count=10, side_lo=24, side_hi=80, seed0=6300)
    s = pm.Phipm("f64pair")
    ops = [pm.DeviceOperator(p_.op) for p_ in probs]
    bs = [[torch.as_tensor(x).cuda() for x in p_.b] for p_ in probs]
    batch = s.batch([p_.t_end for p_ in probs], ops, bs, [p_.tol for p_ in probs], [0] * len(probs))
    rep = batch.autotune()
    ks = [k for k, _ in rep]
    assert ks[0] == 1 and set(ks) <= {1, 2, 4, 8} and len(ks) >= 2
    best = min(rep, key=lambda e: e[1])[0]
    batch.run()
    assert s.last_batched_team() == best
    for p_, u in zip(probs, batch.outs):
        ref, _ = O.phipm(p_.t_end, p_.op, p_.b, p_.tol, 0)
        assert _rel(u, ref) <= 1e-8
    path = tmp_path / "tune.json"
    s.tune_save(path)
    doc = json.loads(path.read_text())
    assert len(doc["batch_entries"]) == 1 and doc["batch_entries"][0]["team"] == best
    assert doc["batch_entries"][0]["log2count"] == 3
    s2 = pm.Phipm("f64pair")
    s2.tune_load(path)
    b2 = s2.batch([p_.t_end for p_ in probs], ops, bs, [p_.tol for p_ in probs], [0] * len(probs))
    b2.run()
    assert s2.last_batched_team() == best
