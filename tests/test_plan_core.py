"""The host planner (plan_core.cpp) on random request sets and launch geometries, built
with the host compiler and run without a GPU (invariants listed in plan_check.cpp), and
planted mistakes in a copy of the planner that the checks must catch."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CORE = os.path.join(ROOT, "paper_1811_11629_gb300", "csrc", "plan_core.cpp")
HARNESS = os.path.join(ROOT, "tests", "plan_check.cpp")


def build_and_run(tmp_path, core_src, cases=3000):
    exe = tmp_path / "plan_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.dirname(CORE), "-o", str(exe),
                    HARNESS, str(core_src)], check=True)
    return subprocess.run([str(exe), str(cases)], capture_output=True, text=True, timeout=600)


def test_planner_invariants(tmp_path):
    out = build_and_run(tmp_path, CORE)
    assert out.returncode == 0, out.stdout[-3000:] + out.stderr[-2000:]
    assert "0 failures" in out.stdout


def test_planner_time_is_linear(tmp_path):
    """32768 instances (the split workload's shape) plan in well under a second; a planner
    that grows its lists per instance instead of geometrically takes seconds here."""
    exe = tmp_path / "plan_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.dirname(CORE), "-o", str(exe),
                    HARNESS, CORE], check=True)
    out = subprocess.run([str(exe), "--time"], capture_output=True, text=True, timeout=300)
    ms = [float(x) for x in out.stdout.split()[1:3]]
    assert max(ms) < 1000.0, out.stdout


MUTANTS = {
    "stride_ignored": ("out += len * stride;", "out += len;"),
    "last_chunk_summed": ("last ? 0 : pieces[k].len", "pieces[k].len"),
    "shortest_first": ("return item_cost[x] > item_cost[y];", "return item_cost[x] < item_cost[y];"),
    "groups_of_strangers": ("&&\n                   hp.items[j].out_off == hp.items[j - 1].out_off + 1)", ")"),
    "segment_drops_tail": ("                    off += l;\n                    left -= l;",
                           "                    left -= l;"),
    "segment_keeps_item": ("out.push_back({c.inst, kNoItem, off, l});",
                           "out.push_back({c.inst, c.item, off, l});"),
    "units_cheapest_first": ("return rx != ry ? rx < ry : unit_cost[x] > unit_cost[y];",
                             "return rx != ry ? rx < ry : unit_cost[x] < unit_cost[y];"),
    "packed_by_cost_not_length": (
        "return hp.items[x].count != hp.items[y].count ? hp.items[x].count > hp.items[y].count\n"
        "                                                          : item_cost[x] > item_cost[y];",
        "return item_cost[x] > item_cost[y];"),
    "packed_groups_cheapest_first": (
        "auto costlier = [&](uint32_t x, uint32_t y) { return unit_cost[x] > unit_cost[y]; };",
        "auto costlier = [&](uint32_t x, uint32_t y) { return unit_cost[x] < unit_cost[y]; };"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_planner_mistake_is_caught(tmp_path, name):
    before, after = MUTANTS[name]
    src = open(CORE).read()
    assert src.count(before) == 1, name
    mutated = tmp_path / "plan_core.cpp"
    mutated.write_text(src.replace(before, after))
    out = build_and_run(tmp_path, mutated, cases=500)
    assert out.returncode != 0, f"the planner checks miss the planted mistake {name}"
