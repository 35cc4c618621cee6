"""Host-side helpers of bench.py: the comment-free source hash that keys the
stored ncu traffic figures."""
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
