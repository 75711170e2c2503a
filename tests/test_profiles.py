"""The profiler summaries under profiles/ give commands that run committed
files only: every `python -m` module exists in the repository, every ncu
command leaves the GPU clocks alone (`--clock-control none`), and no command
names a scratch path."""
import glob
import importlib.util
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands():
    """(file, command text) for every command a summary gives: indented
    blocks of the .md files and the `command` fields of the .json files."""
    out = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        block = []
        for line in open(path).read().splitlines() + [""]:
            if line.startswith("    "):
                block.append(line.strip().rstrip("\\").strip())
            elif block:
                out.append((os.path.basename(path), " ".join(block)))
                block = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.json"))):
        for rec in json.load(open(path)).values():
            if isinstance(rec, dict) and "command" in rec:
                out.append((os.path.basename(path), rec["command"]))
    return out


def test_summaries_give_commands():
    files = {f for f, _ in _commands()}
    assert {"traffic.json", "alu_counts.json", "short_count_kernel_short64.md",
            "fixed_tma_kernel_fixed1k.md"} <= files


def test_commands_run_committed_modules_only():
    for name, cmd in _commands():
        assert "_work/" not in cmd, (name, cmd)
        for mod in re.findall(r"python -m ([\w.]+)", cmd):
            if mod.split(".")[0] in ("pytest",):
                continue
            assert importlib.util.find_spec(mod) is not None, (name, mod)


def test_ncu_commands_leave_the_clocks_alone():
    checked = 0
    for name, cmd in _commands():
        for part in re.split(r"&&|\n", cmd):
            if re.search(r"(^|\s)ncu\s", " " + part):
                assert "--clock-control none" in part, (name, part)
                checked += 1
    assert checked >= 10
