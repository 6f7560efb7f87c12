"""bench.py's --extras selection (host only): every extra the benchmark runs is a known name, "all"
selects each of them, a list selects exactly its members, and unknown names are refused."""

import ast
import os

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_all_selects_every_extra():
    want = bench.extras_selector("all")
    assert all(want(x) for x in bench.EXTRAS)


def test_a_list_selects_exactly_its_members():
    want = bench.extras_selector("tune,cpu")
    assert [x for x in bench.EXTRAS if want(x)] == ["tune", "cpu"]


def test_unknown_extras_are_refused():
    with pytest.raises(ValueError):
        bench.extras_selector("latency,nonsense")


def test_run_extras_asks_for_known_names_only():
    # Every want("...") in run_extras names an entry of EXTRAS, and each entry is asked for.
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    fn = next(n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef) and n.name == "run_extras")
    asked = [c.args[0].value for c in ast.walk(fn)
             if isinstance(c, ast.Call) and isinstance(c.func, ast.Name) and c.func.id == "want"]
    assert sorted(asked) == sorted(bench.EXTRAS)
