"""Repository rules that a test can hold: committed code never reaches into the
untracked working folder, and every profile summary's commands run committed
files only."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tracked():
    try:
        out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True, check=True).stdout
        return [f for f in out.splitlines() if f]
    except (OSError, subprocess.CalledProcessError):  # not a git checkout: walk the tree instead
        files = []
        for d, dirs, names in os.walk(ROOT):
            dirs[:] = [x for x in dirs if not x.startswith((".", "_work", "_build", "gpurun_out", "__pycache__"))]
            files += [os.path.relpath(os.path.join(d, n), ROOT) for n in names]
        return files


def test_no_committed_code_uses_the_working_folder():
    pattern = re.compile(r"[\"'/]_work/")
    for f in _tracked():
        if not f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp", ".sh")) or not os.path.exists(os.path.join(ROOT, f)):
            continue
        if f == "tests/test_repo_hygiene.py":
            continue
        with open(os.path.join(ROOT, f), errors="replace") as fh:
            assert not pattern.search(fh.read()), f


def test_profile_commands_run_committed_files_only():
    tracked = set(_tracked())
    for f in sorted(x for x in tracked if x.startswith("profiles/")):
        with open(os.path.join(ROOT, f), errors="replace") as fh:
            text = fh.read()
        assert "_work" not in text, f
        for block in re.findall(r"```(?:\w*)\n(.*?)```", text, re.S):
            for script in re.findall(r"python3? ([\w/.-]+\.py)", block):
                assert script in tracked, (f, script)
            for mod in re.findall(r"python3? -m ([\w.]+)", block):
                if mod.startswith("paper_1812_07313_gb300"):
                    assert mod.replace(".", "/") + ".py" in tracked, (f, mod)
