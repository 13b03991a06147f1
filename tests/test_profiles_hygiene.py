"""The committed profiling evidence: every ncu command the repository documents
(the summaries under profiles/ and the capture commands of the design notes at
the repository root) leaves the GPU clocks alone (--clock-control none), every
summary gives the command that made it, and profiles/ holds text only (the raw
reports stay out of the repository)."""
import pathlib

ROOT = pathlib.Path(__file__).resolve().parents[1]


def _ncu_commands(text):
    """ncu command lines (after indentation), joined over backslash continuations."""
    lines = text.splitlines()
    out = []
    i = 0
    while i < len(lines):
        line = lines[i].strip()
        if line.startswith("ncu "):
            cmd = line
            while cmd.endswith("\\") and i + 1 < len(lines):
                i += 1
                cmd = cmd[:-1] + " " + lines[i].strip()
            out.append(cmd)
        i += 1
    return out


def _summaries():
    return sorted((ROOT / "profiles").glob("*.md"))


def test_every_documented_ncu_command_keeps_the_clocks():
    notes = ROOT / "DESIGN.md"
    cmds = [(f.name, c) for f in _summaries() + [notes] for c in _ncu_commands(f.read_text())]
    assert cmds
    for name, cmd in cmds:
        assert "--clock-control none" in cmd, (name, cmd)


def test_every_profile_summary_gives_its_command():
    assert _summaries()
    for f in _summaries():
        assert _ncu_commands(f.read_text()), f.name


def test_profiles_hold_text_only():
    for f in (ROOT / "profiles").iterdir():
        assert f.suffix in (".md", ".txt"), f.name
