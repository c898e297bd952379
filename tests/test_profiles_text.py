"""The ncu summaries under profiles/: plain text only, every ncu command
they give runs with the GPU clocks left alone (--clock-control none), and the
commands run committed files only (no scratch scripts)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _commands(text):
    """Logical shell commands of a summary: indented lines, backslash continuations joined."""
    out, cur = [], ""
    for line in text.splitlines():
        if not line.startswith("    "):
            if cur:
                out.append(cur)
            cur = ""
            continue
        cur += " " + line.strip().rstrip("\\")
        if not line.rstrip().endswith("\\"):
            out.append(cur)
            cur = ""
    if cur:
        out.append(cur)
    return out


def test_profiles_hold_text_only():
    for name in os.listdir(PROFILES):
        assert os.path.splitext(name)[1] in (".md", ".txt", ".json"), name


def test_every_ncu_command_leaves_the_clocks_alone():
    seen = 0
    for name in sorted(os.listdir(PROFILES)):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(PROFILES, name)) as f:
            for cmd in _commands(f.read()):
                for part in re.split(r"&&|;", cmd):
                    if re.match(r"\s*ncu\s", part):
                        seen += 1
                        assert "--clock-control none" in part, f"{name}: {part.strip()[:80]}"
    assert seen >= 5


def test_commands_run_committed_files_only():
    for name in sorted(os.listdir(PROFILES)):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(PROFILES, name)) as f:
            for cmd in _commands(f.read()):
                assert "_work" not in cmd, f"{name}: {cmd.strip()[:80]}"
                for script in re.findall(r"python3? (\S+\.py)", cmd):
                    assert os.path.exists(os.path.join(ROOT, script)), f"{name}: {script}"
