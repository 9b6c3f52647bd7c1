"""Static checks of the separation between the CUDA path and the oracle.

The oracle (oracle/) is test infrastructure: the library and its binding
(paper_2310_13908_gb300/) never import, include or load it, and the oracle
never uses the library. Both take their inputs from capsule_inputs/, which
imports neither. Nothing in the repository uses the untracked working folder.
"""

import ast
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PACKAGE = "paper_2310_13908_gb300"


def _files(folder, exts):
    out = []
    for dirpath, dirnames, filenames in os.walk(os.path.join(ROOT, folder)):
        dirnames[:] = [d for d in dirnames if d not in ("__pycache__", "_build")]
        out += [os.path.join(dirpath, f) for f in filenames if f.endswith(exts)]
    return sorted(out)


def _imported_modules(path):
    tree = ast.parse(open(path).read(), filename=path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                mods.add(node.module.split(".")[0])
        elif isinstance(node, ast.Call) and getattr(node.func, "attr", "") == "import_module":
            if node.args and isinstance(node.args[0], ast.Constant):
                mods.add(str(node.args[0].value).split(".")[0])
    return mods


def test_library_never_uses_the_oracle():
    for path in _files(PACKAGE, (".py",)):
        assert "oracle" not in _imported_modules(path), path
        text = open(path).read()
        assert "liboracle" not in text and "stokes_oracle" not in text, path
    for path in _files(os.path.join(PACKAGE, "csrc"), (".cu", ".cuh", ".h", ".cpp")):
        for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', open(path).read()):
            assert "oracle" not in inc, (path, inc)


def test_oracle_never_uses_the_library():
    for path in _files("oracle", (".py",)):
        assert PACKAGE not in _imported_modules(path), path
        text = open(path).read()
        assert "libstokesreg" not in text and "csrc" not in text, path
    for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]',
                          open(os.path.join(ROOT, "oracle", "stokes_oracle.c")).read()):
        assert inc in ("math.h", "stdint.h", "stddef.h", "stdlib.h", "string.h", "omp.h"), inc


def test_input_generators_import_neither_side():
    for path in _files("capsule_inputs", (".py",)):
        mods = _imported_modules(path)
        assert "oracle" not in mods and PACKAGE not in mods, (path, mods)


def test_nothing_committed_uses_the_work_folder():
    try:
        tracked = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True,
                                 check=True).stdout.split()
    except (OSError, subprocess.CalledProcessError):
        pytest.skip("not a git checkout")
    pattern = re.compile(r"(^|[\s\"'/(=])_work/")
    for rel in tracked:
        if rel == ".gitignore" or not rel.endswith((".py", ".cu", ".cuh", ".h", ".c", ".sh", ".txt")):
            continue
        path = os.path.join(ROOT, rel)
        if not os.path.isfile(path):
            continue
        for n, line in enumerate(open(path, errors="replace"), 1):
            assert not pattern.search(line), f"{rel}:{n}: {line.strip()}"
