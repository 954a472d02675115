"""The command line (python -m paper_2607_00981_gb300) on the host simulation of the
library's plans: JSON lines per iteration, checkpoint at the end and resume from it."""
import json

import paper_2607_00981_gb300 as pkg
from paper_2607_00981_gb300 import __main__ as cli

from ._helpers import hostsim_lib


def test_iterations_checkpoint_and_resume(monkeypatch, capsys, tmp_path):
    monkeypatch.setattr(pkg, "load", hostsim_lib)
    ck = tmp_path / "o3v12.ck"
    assert cli.main(["--workload", "o3v12", "--iters", "3", "--checkpoint", str(ck)]) == 0
    lines = [json.loads(x) for x in capsys.readouterr().out.splitlines()]
    assert [x["iter"] for x in lines] == [1, 2, 3]
    assert lines[0]["delta_e"] is None and lines[1]["delta_e"] == lines[1]["energy"] - lines[0]["energy"]
    assert set(lines[0]["step_ms"]) >= {"pp", "ring", "hh", "update"}
    # resuming continues the sequence: its first iteration equals a fourth one
    assert cli.main(["--workload", "o3v12", "--iters", "1", "--resume", str(ck)]) == 0
    resumed = json.loads(capsys.readouterr().out.splitlines()[0])
    assert cli.main(["--workload", "o3v12", "--iters", "4"]) == 0
    straight = [json.loads(x) for x in capsys.readouterr().out.splitlines()]
    assert resumed["energy"] == straight[3]["energy"] and resumed["r"] == straight[3]["r"]


import pytest  # noqa: E402


@pytest.mark.gpu
def test_t4_passes_print_one_line_per_pass(capsys):
    """--t4 o,v times the compact-T4 ladder and post-processing on the GPU; the norm of
    the post-processed R4 is the same in every pass (same inputs, deterministic)."""
    assert cli.main(["--t4", "2,12", "--precision", "bf16x3", "--reps", "2"]) == 0
    lines = [json.loads(x) for x in capsys.readouterr().out.splitlines()]
    assert [x["pass"] for x in lines] == [0, 1]
    assert lines[0]["n4"] == 5 and lines[0]["r4_norm"] > 0
    assert lines[0]["r4_norm"] == lines[1]["r4_norm"]
    assert all(x["ladder_ms"] > 0 and x["post_ms"] > 0 for x in lines)


@pytest.mark.gpu
def test_batch_launches_one_line(capsys):
    """--batch o,v,n runs n identical instances in one graph and prints its launch times."""
    assert cli.main(["--batch", "3,12,4", "--iters", "2", "--precision", "bf16x3"]) == 0
    line = json.loads(capsys.readouterr().out.splitlines()[-1])
    assert line["batch"] == [3, 12, 4] and len(line["launch_ms"]) == 2 and line["kernels"] > 0
