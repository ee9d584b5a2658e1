"""Source hygiene of the product: the library package never reaches the
oracle (no CPU fallback), nothing committed refers to scratch files or to
paths outside the repository, and no source names the batched-copy runtime
calls, which the GPU pool rejects."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PACKAGE = os.path.join(ROOT, "paper_2410_01754_gb300")
SOURCE_EXT = (".py", ".cu", ".cpp", ".c", ".h", ".cuh", ".sh")


def _sources(*tops):
    for top in tops:
        if os.path.isfile(top):
            yield top
            continue
        for d, dirs, files in os.walk(top):
            dirs[:] = [x for x in dirs if x not in ("__pycache__", "golden")]
            for f in files:
                if f.endswith(SOURCE_EXT):
                    yield os.path.join(d, f)


def _read(p):
    with open(p, encoding="utf-8", errors="replace") as fh:
        return fh.read()


def test_library_never_imports_the_oracle():
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|liboracle", re.M)
    bad = [p for p in _sources(PACKAGE) if pat.search(_read(p))]
    assert not bad, bad


def test_no_scratch_or_outside_paths():
    scratch = "_" + "work" + "/"
    outside = "/root/" + "reference"
    tops = [PACKAGE] + [os.path.join(ROOT, d) for d in ("oracle", "synth", "include", "tests")]
    tops += [os.path.join(ROOT, f) for f in ("bench.py", "__graft_entry__.py")]
    bad = [p for p in _sources(*tops) if scratch in _read(p) or outside in _read(p)]
    assert not bad, bad


def test_no_batched_copy_calls():
    names = [pre + "Memcpy" + mid + "Batch" + "Async" for pre in ("cuda", "cu") for mid in ("", "3D")]
    tops = [PACKAGE] + [os.path.join(ROOT, d) for d in ("oracle", "synth", "include", "tests")]
    tops += [os.path.join(ROOT, f) for f in ("bench.py", "__graft_entry__.py")]
    bad = [(p, n) for p in _sources(*tops) for n in names if n in _read(p)]
    assert not bad, bad
