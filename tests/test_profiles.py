"""The committed ncu summaries: each gives the full command that made it,
the command runs committed files only (bench.py, the package), and every ncu
command leaves the GPU clocks alone (--clock-control none).  No GPU."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands(text):
    """The inline code spans (odd segments between backticks) that run ncu."""
    spans = text.split("`")[1::2]
    return [c for c in spans if re.search(r"(^|\s)ncu\s+-", c)]


def test_every_summary_has_a_committed_command():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert files
    for path in files:
        cmds = _commands(open(path).read())
        assert cmds, path
        for c in cmds:
            assert "--clock-control none" in c, (path, c)
            assert "_work" not in c and "/root/" not in c, (path, c)
            for script in re.findall(r"python\s+(\S+\.py)", c):
                assert os.path.exists(os.path.join(ROOT, script)), (path, script)
