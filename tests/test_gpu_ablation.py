"""The split ablation tool (Sections 4.1 and 5 of the paper on synthetic
graphs): every split variant leaves no internally disconnected community and
the variants agree on the modularity."""
import json

import pytest

pytestmark = pytest.mark.gpu


def test_ablation_on_planted(capsys):
    from paper_2402_11454_gb300 import ablation
    assert ablation.main(["--workloads", "planted", "--steps", "1"]) == 0
    rows = [json.loads(line) for line in capsys.readouterr().out.splitlines() if line.startswith("{")]
    assert len(rows) == len(ablation.VARIANTS)
    qs = []
    for r in rows:
        assert r["workload"] == "planted" and r["ms"] > 0
        if r["split"] != "none":
            assert r["disconnected"] == 0
            if not r["refine"]:
                qs.append(r["modularity"])
    # every split technique yields the same labels; pass and last differ in where the split runs
    assert max(qs) - min(qs) < 2e-3
