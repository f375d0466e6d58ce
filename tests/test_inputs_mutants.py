"""The input generators' pins reject a generator with a planted mistake.

The seeded generators (paper_2104_02646_gb300/inputs.py) feed both the CUDA
path and the oracle, so parity cannot see a mistake in them; their own pins
(tests/test_inputs.py and the workload pins of tests/test_oracle_pins.py) must.
Each case copies inputs.py, plants one mistake, registers the copy as
paper_2104_02646_gb300.inputs before those pins import it, and requires a
failing pin; an unchanged copy must pass them.  The committed generator is
never modified.  CPU only."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2104_02646_gb300", "inputs.py")
PINS = [os.path.join(ROOT, "tests", "test_inputs.py"),
        os.path.join(ROOT, "tests", "test_oracle_pins.py") + "::test_block_inputs_are_conforming_and_positive",
        os.path.join(ROOT, "tests", "test_oracle_pins.py") + "::test_workload_counts"]

MUTANTS = {
    # every cell split the same way (no mirror on alternate cells): faces no longer conform
    "split_not_mirrored": ("tets[sel] = corner_nodes[sel][:, _SPLIT_ORIENTED[p]]",
                           "tets[sel] = corner_nodes[sel][:, _SPLIT_ORIENTED[0]]"),
    # the second triangle of each cloth cell wound the other way
    "cloth_triangle_flipped": ("tris[1::2] = np.stack([a, d, c], axis=1)", "tris[1::2] = np.stack([a, c, d], axis=1)"),
    # the hinge's wing tips swapped
    "hinge_wings_swapped": ("out = np.stack([o[h1], o[h2], p[h1], q[h1]], axis=1)",
                            "out = np.stack([o[h2], o[h1], p[h1], q[h1]], axis=1)"),
    # block64's Poisson ratios drawn from a wider range
    "block_nu_range": ("nu = rng.uniform(0.2, 0.45, E)", "nu = rng.uniform(0.2, 0.49, E)"),
    # Poisson arrivals with the rate where the mean gap belongs
    "query_rate_inverted": ("t += rng.exponential(1.0 / rate)", "t += rng.exponential(rate)"),
    # batch element-count targets over a range ten times too wide
    "batch_target_range": ("target = math.exp(rng.uniform(math.log(lo), math.log(hi)))",
                           "target = math.exp(rng.uniform(math.log(lo), math.log(10 * hi)))"),
    # Lame lambda with (1 - nu) for (1 - 2 nu)
    "lame_lambda": ("E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))", "E * nu / ((1.0 + nu) * (1.0 - nu))"),
}

_BOOT = """
import importlib.util, sys
root, path = sys.argv[1:3]
sys.path.insert(0, root)
import paper_2104_02646_gb300 as pkg
spec = importlib.util.spec_from_file_location("paper_2104_02646_gb300.inputs", path)
mod = importlib.util.module_from_spec(spec)
sys.modules["paper_2104_02646_gb300.inputs"] = mod
spec.loader.exec_module(mod)
pkg.inputs = mod
import pytest
sys.exit(pytest.main(sys.argv[3:] + ["-x", "-q", "-p", "no:cacheprovider"]))
"""


def _pins(tmp_path, name, text=None, repl=None):
    src = open(SRC).read()
    if text is not None:
        assert src.count(text) == 1, name
        src = src.replace(text, repl)
    path = tmp_path / f"{name}.py"
    path.write_text(src)
    cmd = [sys.executable, "-c", _BOOT, ROOT, str(path)] + PINS
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = tmp_path_factory.mktemp("inputs_mutants")
    jobs = {"unchanged": lambda: _pins(base, "unchanged")}
    for name, (text, repl) in MUTANTS.items():
        jobs[name] = lambda n=name, t=text, r=repl: _pins(base, n, t, r)
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futures = {k: ex.submit(f) for k, f in jobs.items()}
        return {k: f.result() for k, f in futures.items()}


def test_unchanged_copy_passes_the_pins(outcomes):
    assert outcomes["unchanged"].returncode == 0, outcomes["unchanged"].stdout[-3000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(outcomes, name):
    r = outcomes[name]
    assert r.returncode == 1 and "failed" in r.stdout, (name, r.returncode, r.stdout[-3000:])
