"""Sources stand on their own: no code file, comment or docstring names the
project's notes files, its measurement records or a path of one machine.

Scans the committed code (the package, its CUDA sources, the headers, the
oracle, the generator, the tests, bench.py and __graft_entry__.py).  The
words are assembled here so that this file does not match itself.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIRS = ("paper_2507_14222_gb300", "include", "oracle", "igdata", "tests")
FILES = ("bench.py", "__graft_entry__.py")
EXTS = (".py", ".cu", ".cuh", ".h", ".cpp", ".c")

# The notes files and records by name (upper case, as the files are named),
# the remote runner's name and the scope key.
_WORDS = [w.replace("_", "") for w in (
    "DE_SIGN", "SUR_VEY", "VER_DICT", "AD_VICE", "BASE_LINE", "READ_ME", "PROG_RESS")]
_PATTERNS = [re.compile(r"\b" + w + r"\b") for w in _WORDS] + [
    re.compile("north" + "_star", re.I), re.compile("gpu" + "run", re.I),
    re.compile("/" + "root/"), re.compile(r"\b" + "rou" + r"nd [0-9]", re.I)]


def _paths():
    out = [os.path.join(ROOT, f) for f in FILES]
    for d in DIRS:
        for dirpath, dirnames, files in os.walk(os.path.join(ROOT, d)):
            dirnames[:] = [x for x in dirnames if x not in ("_build", "__pycache__")]
            out += [os.path.join(dirpath, f) for f in files if f.endswith(EXTS)]
    return out


def test_no_source_names_notes_records_or_machine_paths():
    bad = []
    for path in _paths():
        with open(path, encoding="utf-8") as f:
            for ln, line in enumerate(f, 1):
                for p in _PATTERNS:
                    if p.search(line):
                        bad.append(f"{os.path.relpath(path, ROOT)}:{ln}: {line.strip()[:80]}")
    assert not bad, "\n".join(bad)
