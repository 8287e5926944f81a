"""The oracle's pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle/gpz_oracle.cpp: a wrong
sign, a dropped term, a wrong index, swapped operands, or an off-by-one.
These are the mistakes a restatement of Sections 4.1-4.3 could plausibly
contain.  The copy is compiled on the CPU and the pins of
tests/test_oracle_pins.py run against it (GPZ_ORACLE_LIB points the oracle's
loader at the copy).  Every mutant must fail at least one pin through an
assertion; an unmutated copy, built the same way, must pass them all.
Nothing here touches a GPU."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from oracle import build as oracle_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (what the mistake is, the text it replaces, the mistaken text)
MUTANTS = [
    ("reconstruction steps downwards from the block minimum (Section 4.1)",
     "return std::fmaf((float)q, s, boundary_min);",
     "return std::fmaf((float)q, -s, boundary_min);"),
    ("verification threshold rounded above eb instead of below",
     "eb * (1.0 - std::ldexp(1.0, -22))",
     "eb * (1.0 + std::ldexp(1.0, -22))"),
    ("relative bound taken from the maximum alone (range term dropped)",
     "double range = (double)hi - (double)lo;",
     "double range = (double)hi;"),
    ("segId and segOffset swapped (remainder used as the id)",
     "st->seg_id[f][i] = st->q[f][i] / m;",
     "st->seg_id[f][i] = st->q[f][i] % m;"),
    ("axes linearised in reverse order (Section 4.1)",
     "k = k * (1u << st->g[f]) + st->seg_id[f][i];",
     "k = k * (1u << st->g[f]) + st->seg_id[P - 1 - f][i];"),
    ("run boundaries found in storage order instead of sorted order (Section 4.3)",
     "(id != st->key[st->perm[j - 1]])",
     "(id != st->key[j - 1])"),
    ("delta of the unique ids off by one (Section 4.3)",
     "st->uniq[k] - st->uniq[k - 1];",
     "st->uniq[k] - st->uniq[k - 1] - 1;"),
    ("fixed-length codes packed most significant bit first",
     "if ((v >> b) & 1u) words[t / 32] |= 1u << (t % 32);",
     "if ((v >> b) & 1u) words[t / 32] |= 1u << (31 - t % 32);"),
    ("decoder forgets to accumulate the deltas",
     "uint64_t id = (k == 0) ? delta : (uint64_t)uniq[k - 1] + delta;",
     "uint64_t id = delta;"),
]


def _build_copy(tmp_path, name, old, new):
    src = open(oracle_build.SRC).read()
    if old is not None:
        assert src.count(old) == 1, "mutation site not unique: %r" % old
        src = src.replace(old, new)
    cpp = tmp_path / (name + ".cpp")
    cpp.write_text(src)
    so = tmp_path / (name + ".so")
    subprocess.run(["g++"] + oracle_build.CXXFLAGS + ["-I", os.path.dirname(oracle_build.SRC), str(cpp),
                    "-o", str(so)], check=True, capture_output=True, timeout=600)
    return str(so)


def _run_pins(lib):
    env = dict(os.environ, GPZ_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout + r.stderr


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    tmp = tmp_path_factory.mktemp("mutants")
    jobs = [("control", None, None)] + [("m%d" % i, old, new) for i, (_, old, new) in enumerate(MUTANTS)]
    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1)) as ex:
        libs = list(ex.map(lambda j: _build_copy(tmp, *j), jobs))
        results = list(ex.map(_run_pins, libs))
    return dict(zip([j[0] for j in jobs], results))


def test_unmutated_copy_passes_the_pins(outcomes):
    rc, out = outcomes["control"]
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("i", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_mistake(outcomes, i):
    rc, out = outcomes["m%d" % i]
    # exit code 1 is pytest's "some tests failed": a pin's assertion, not a crash
    assert rc == 1 and " failed" in out, (MUTANTS[i][0], rc, out[-2000:])
