"""Checked mode's bounds predicates (paper_2604_02586_b300/csrc/checks.h),
compiled for the host and exercised without a GPU.

The kernels call the same inline functions before every index they take from
data (a (record, tile) item's tile and list slot, tile ranges, the moment
origin's pixel, a list entry's Gaussian); here each predicate is checked at and
around its edges."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_02586_b300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "checks.h"
using namespace tsp;
static int fails = 0;
#define EXPECT(c) do { if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); ++fails; } } while (0)
int main() {
    EXPECT(index_ok(0, 1));
    EXPECT(!index_ok(1, 1));
    EXPECT(!index_ok(0, 0));
    EXPECT(index_ok(4294967294ull, 4294967295ull));
    EXPECT(!index_ok(0xffffffffull, 0xffffffffull));
    EXPECT(range_ok(3, 3, 3));
    EXPECT(range_ok(0, 5, 5));
    EXPECT(!range_ok(4, 3, 10));      // not ascending
    EXPECT(!range_ok(2, 11, 10));     // past the buffer
    EXPECT(slot_ok(10, 0, 11));       // one-element list, slot 0
    EXPECT(!slot_ok(10, 1, 11));      // slot past its end
    EXPECT(!slot_ok(10, 0, 10));      // empty list
    EXPECT(!slot_ok(12, 0, 10));      // inverted list
    EXPECT(pixel_ok(0, 1, 1));
    EXPECT(!pixel_ok(1, 1, 1));
    EXPECT(pixel_ok(8191ull * 8192ull + 8191ull, 8192, 8192));
    EXPECT(!pixel_ok(8192ull * 8192ull, 8192, 8192));
    EXPECT(!pixel_ok(0, 0, 5));
    for (unsigned s = 1; s < kSiteCount; ++s) EXPECT(check_site_name(s)[0] != 'u');
    EXPECT(check_site_name(kSiteCount)[0] == 'u');
    std::printf("%d\n", fails);
    return fails != 0;
}
"""


def test_bounds_predicates_on_the_host(tmp_path):
    src = tmp_path / "checks_test.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "checks_test"
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Werror", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout


def test_checked_option_is_in_the_abi():
    import ctypes as C
    import paper_2604_02586_b300 as tsp
    from paper_2604_02586_b300 import build as tbuild
    tbuild.build()
    o = tsp.Options()
    assert tsp.lib().tsp_default_options(C.byref(o)) == tsp.TSP.OK
    assert o.checked == 0
