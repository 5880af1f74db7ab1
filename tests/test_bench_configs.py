"""bench_configs/*.json: every file names only bench.py options, parses into the workload it
describes, and an option given on the command line overrides the file."""
import glob
import json
import os

import pytest

import bench

FILES = sorted(glob.glob(os.path.join(bench.ROOT, "bench_configs", "*.json")))


def test_the_five_configurations_are_there():
    names = {os.path.basename(f)[:-5] for f in FILES}
    assert names == {"d2q9_channel_disk", "d2q9_sedimentation", "d3q19_suspension_512", "d3q19_ensemble_64",
                     "d3q19_closure"}


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f) for f in FILES])
def test_file_parses_into_its_options(path):
    cfg = json.load(open(path))
    assert isinstance(cfg.get("description"), str) and cfg["description"]
    args = bench.parse(["--config", path])
    for k, v in cfg.items():
        if k != "description":
            assert getattr(args, k) == v, k
    if args.workload not in ("ensemble_64", "closure"):
        wl = bench.workload(args)
        assert wl.lattice == ("D2Q9" if args.workload.startswith("d2q9") else "D3Q19")


def test_command_line_wins():
    path = os.path.join(bench.ROOT, "bench_configs", "d3q19_suspension_512.json")
    args = bench.parse(["--config", path, "--steps", "7", "--precision", "fp16"])
    assert args.steps == 7 and args.precision == "fp16" and args.workload == "d3q19_512"


def test_unknown_key_is_refused(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text(json.dumps({"workload": "d3q19_512", "no_such_option": 1}))
    with pytest.raises(SystemExit):
        bench.parse(["--config", str(p)])
