"""The committed ncu summaries under profiles/ follow the capture rules: each
names the command that made it, every ncu invocation leaves the GPU clocks
alone (--clock-control none), and what the commands run exists in the
repository."""
import glob
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands(text):
    """Shell commands of the fenced code blocks (continuation lines joined)
    and of inline code spans."""
    out = [c.strip() for c in re.findall(r"`([^`\n]*(?:ncu|python)\s[^`\n]*)`", text)]
    for block in re.findall(r"```[a-z]*\n(.*?)```", text, flags=re.S):
        cmd = ""
        for line in block.splitlines():
            cmd += line.rstrip("\\").strip() + " "
            if not line.rstrip().endswith("\\"):
                if cmd.strip():
                    out.append(cmd.strip())
                cmd = ""
    return out


def _summaries():
    return [p for p in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))) if not p.endswith("README.md")]


def test_every_summary_names_its_ncu_command():
    assert len(_summaries()) >= 5
    for path in _summaries():
        cmds = [c for c in _commands(open(path).read()) if re.search(r"(^|[\s;&(])ncu\s", c)]
        assert cmds, f"{os.path.basename(path)} gives no ncu command"
        for c in cmds:
            for inv in re.split(r"&&|;", c):
                if re.search(r"(^|\s)ncu\s", inv):
                    assert "--clock-control none" in inv, (os.path.basename(path), inv)


def test_commands_run_committed_files():
    texts = [open(p).read() for p in _summaries()]
    rec = json.load(open(os.path.join(ROOT, "profiles", "herk_tc_traffic.json")))
    assert "--clock-control none" in rec["command"]
    texts.append("```\n" + rec["command"] + "\n```\n")
    for text in texts:
        for c in _commands(text):
            for mod in re.findall(r"python -m (paper_1307_8052_gb300\.\w+)", c):
                assert os.path.exists(os.path.join(ROOT, *mod.split(".")) + ".py"), mod
            for script in re.findall(r"python (\S+\.py)", c):
                assert os.path.exists(os.path.join(ROOT, script)), script
                assert not script.startswith("_work"), script
            # the bench options a command uses are options bench.py has
            for run in re.findall(r"python bench\.py([^&;]*)", c):
                src = open(os.path.join(ROOT, "bench.py")).read()
                for flag in re.findall(r"(--[a-z0-9-]+)", run):
                    assert f'"{flag}"' in src, flag
