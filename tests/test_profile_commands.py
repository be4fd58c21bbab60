"""The ncu summaries under profiles/ give the commands their figures came
from.  Every `python bench.py ...` command in them (continuation lines and
shell variables such as F="..." resolved) must use only options that
bench.py still accepts, so that each command can be run again as written."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _bench_options() -> set[str]:
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"],
                         capture_output=True, text=True, check=True).stdout
    return set(re.findall(r"(--[a-z0-9][a-z0-9-]*)", out))


def _commands(text: str) -> list[str]:
    """bench.py command lines of one summary, with continuations joined and
    $NAME variables (NAME="..." lines of the same file) expanded."""
    lines = text.splitlines()
    joined, cur = [], ""
    for ln in lines:
        s = ln.strip()
        if cur:
            cur += " " + s.rstrip("\\").strip()
            if not s.endswith("\\"):
                joined.append(cur)
                cur = ""
        elif s.endswith("\\"):
            cur = s.rstrip("\\").strip()
        else:
            joined.append(s)
    if cur:
        joined.append(cur)
    env = {}
    for s in joined:
        m = re.fullmatch(r'([A-Z][A-Z0-9_]*)="([^"]*)"', s)
        if m:
            env[m.group(1)] = m.group(2)
    cmds = []
    for s in joined:
        if "python bench.py" not in s or s.startswith(("|", "-", "*")) or "`" in s:
            continue
        for name, val in env.items():
            s = s.replace("$" + name, val)
        cmds.append(s[s.index("python bench.py"):])
    return cmds


def test_every_profile_command_uses_options_bench_accepts():
    known = _bench_options()
    assert "--workload" in known and "--no-pfb" in known
    checked = 0
    for name in sorted(os.listdir(PROFILES)):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(PROFILES, name)) as f:
            text = f.read()
        for cmd in _commands(text):
            assert "$" not in cmd, f"{name}: unresolved variable in {cmd!r}"
            used = set(re.findall(r"(?<![\w-])(--[a-z0-9][a-z0-9-]*)", cmd))
            unknown = used - known
            assert not unknown, f"{name}: {sorted(unknown)} not accepted by bench.py in {cmd!r}"
            checked += 1
    assert checked >= 10


def test_command_parser_joins_continuations_and_expands_variables():
    text = ('    F="--no-cpu --no-sweep"\n'
            '    ncu --metrics a \\\n'
            '        --clock-control none python bench.py $F --steps 1 \\\n'
            '        --warmup 1\n')
    assert _commands(text) == ["python bench.py --no-cpu --no-sweep --steps 1 --warmup 1"]
