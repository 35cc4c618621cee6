"""Host-side helpers of bench.py: the comment-free source hash that keys the
stored ncu traffic figures, and the summary of the clocks sampled during the
timed region."""
import bench


def test_strip_c_comments_keeps_code_and_literals():
    src = ('int a = 1; // trailing\n'
           '/* block\n   comment */ int b = 2;\n'
           '\n'
           'asm("ld.global.nc.u16 %0, [%1]; // not a comment" : "=h"(x));\n'
           "char c = '/'; char d = '\\''; /**/int e;   \n")
    out = bench.strip_c_comments(src)
    assert out.splitlines() == [
        "int a = 1;",
        "  int b = 2;",
        'asm("ld.global.nc.u16 %0, [%1]; // not a comment" : "=h"(x));',
        "char c = '/'; char d = '\\'';  int e;",
    ]


def test_comment_edits_keep_the_hash_and_code_edits_change_it():
    base = "__global__ void k(float* p) { p[0] = 1.f; }\n"
    commented = "// kernel\n/* two\n   lines */\n__global__ void k(float* p) { p[0] = 1.f; } // end\n\n"
    changed = "__global__ void k(float* p) { p[0] = 2.f; }\n"
    assert bench.strip_c_comments(base) == bench.strip_c_comments(commented)
    assert bench.strip_c_comments(base) != bench.strip_c_comments(changed)


def test_clock_summary_reports_median_clock_and_throttle_reasons():
    """The clocks record of a bench line: median SM clock under load, the
    maximum clock, and every throttle reason seen active (a run that saw a
    thermal or hardware slowdown is to be rejected, power capping is noted)."""
    lines = [
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1400.0, 0x0000000000000040, Not Active, Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = bench.ClockSampler.summarise(lines)
    assert s["sm_mhz"] == 2040 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.ClockSampler.summarise([])["sm_mhz"] is None
