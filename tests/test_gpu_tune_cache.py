"""The persisted choice of kernel forms (POISSON_TUNE_CACHE): a plan created with the variable
set writes its timed choice to the file, and a later process that finds its shape in the
file takes the recorded forms without timing them.  Each step runs in its own process so
that the in-process decisions of the other tests do not interfere."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, %r)
import torch
from paper_1612_01799_gb300 import Plan
torch.cuda.set_device(0)
with Plan(%d, 10.0, 1e-6, "f32") as p:
    print(json.dumps({"z": p.z_form, "y": p.y_form, "x": p.x_form, "xy": p.xy_form,
                      "name": torch.cuda.get_device_name(0)}))
"""


def child(path, N):
    env = dict(os.environ, POISSON_TUNE_CACHE=str(path))
    r = subprocess.run([sys.executable, "-c", CHILD % (ROOT, N)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01799_gb300 import build
    build.build()


def test_choice_is_written_and_read_back(built, tmp_path):
    path = tmp_path / "tune.txt"
    first = child(path, 128)
    lines = path.read_text().splitlines()
    assert lines[0] == "gspoisson-tune 1"
    rec = lines[1].split(" ", 7)
    assert [int(v) for v in rec[:7]] == [128, 0, first["z"], first["y"], first["x"], first["xy"], 0]
    assert rec[7] == first["name"]
    # A recorded choice that timing would not make at N = 128 (every pass in its block form):
    # the next process takes it as recorded.
    path.write_text("gspoisson-tune 1\n128 0 0 0 0 0 0 %s\n" % first["name"])
    again = child(path, 128)
    assert (again["z"], again["y"], again["x"], again["xy"]) == (0, 0, 0, 0)
    assert path.read_text().count("\n") == 2                 # nothing new appended


def test_invalid_lines_are_ignored(built, tmp_path):
    path = tmp_path / "tune.txt"
    path.write_text("gspoisson-tune 1\n128 0 7 0 0 0 0 SomeGPU\n128 0 0 0 0 0 1 SomeGPU\ngarbage\n")
    got = child(path, 128)
    assert got["z"] in (0, 1, 2)
    assert path.read_text().splitlines()[-1].startswith("128 0 ")
