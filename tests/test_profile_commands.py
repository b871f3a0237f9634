"""The commands recorded in the profile summaries stay runnable: every
``python bench.py`` invocation uses only options the benchmark defines, and
every ncu command leaves the GPU clocks alone (``--clock-control none``)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _commands():
    """(file, command) for each shell command in a fenced block, continuation lines joined."""
    out = []
    for f in sorted(os.listdir(PROFILES)):
        if not f.endswith(".md"):
            continue
        text = open(os.path.join(PROFILES, f)).read()
        for block in re.findall(r"```[a-z]*\n(.*?)```", text, flags=re.S):
            joined = re.sub(r"\\\n\s*", " ", block)
            out += [(f, ln.strip()) for ln in joined.splitlines() if ln.strip()]
    return out


def _bench_options():
    src = open(os.path.join(ROOT, "bench.py")).read()
    return set(re.findall(r'add_argument\(\s*"(--[a-z0-9-]+)"', src))


def test_profiles_record_commands():
    files = [f for f in os.listdir(PROFILES) if f.endswith(".md")]
    assert files
    have = {f for f, _ in _commands()}
    assert have == set(files), set(files) - have


def test_bench_options_in_profile_commands_exist():
    opts = _bench_options()
    assert "--steps" in opts and "--only" in opts
    for f, cmd in _commands():
        for part in re.split(r"&&|;", cmd):
            if "bench.py" not in part:
                continue
            tail = part.split("bench.py", 1)[1]
            tail = re.split(r"\s[12]?>", tail)[0]           # drop redirections
            used = set(re.findall(r"(?<!\S)(--[a-z0-9-]+)", tail))
            assert used <= opts, (f, sorted(used - opts))


def test_ncu_commands_leave_clocks_alone():
    n = 0
    for f, cmd in _commands():
        for part in re.split(r"&&|;", cmd):
            if re.match(r"\s*ncu\s", part):
                n += 1
                assert "--clock-control none" in part, (f, part)
    assert n > 0
