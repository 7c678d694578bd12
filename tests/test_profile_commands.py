"""Every bench.py command quoted in profiles/ (the commands the ncu summaries were made with)
parses with bench.py's own argument parser, so a summary never cites an option the bench no
longer has."""
from __future__ import annotations

import glob
import json
import os
import re
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands():
    out = []
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*"))):
        text = open(path).read()
        if path.endswith(".json"):
            text = json.load(open(path)).get("command", "")
        for m in re.finditer(r"python bench\.py([^\"\n`]*)", text):
            args = m.group(1).strip()
            alts = re.search(r"<([^>]+)>", args)
            if alts:                               # a placeholder of alternatives: each one
                for a in alts.group(1).split("|"):
                    out.append((os.path.basename(path), args.replace(alts.group(0), a)))
            else:
                out.append((os.path.basename(path), args))
    return out


COMMANDS = _commands()


def test_profiles_quote_bench_commands():
    assert len(COMMANDS) >= 6


@pytest.mark.parametrize("where,args", COMMANDS, ids=[f"{w}:{a}" for w, a in COMMANDS])
def test_profile_command_parses(where, args):
    sys.path.insert(0, ROOT)
    import bench
    ns = bench.build_parser().parse_args(shlex.split(args))
    assert ns.gpus == 1, where                      # profiles are single-GPU captures
