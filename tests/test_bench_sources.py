"""Host logic of the benchmark's source hash (CPU only).

The benchmark reports the double-float kernel's executed flops, FP32
instructions and DRAM traffic per cell from constants taken with ncu, and only
while the kernel sources hash to the value they were taken at; the hash ignores
comments and blank lines, so that rewording a comment keeps the constants while
any change to the code drops them (the roofline then reports no achieved rate).
"""
import bench


def test_comments_and_blank_lines_are_dropped():
    src = ("int a = 1;  // one\n"
           "\n"
           "/* block\n   comment */ int b = 2;   \n"
           "    \n"
           "float c = a / b; /* tail */\n")
    assert bench.code_of(src) == "int a = 1;\n int b = 2;\nfloat c = a / b;"


def test_literals_keep_comment_markers():
    src = ('const char* s = "http://x /* y */";\n'
           "char q = '\"'; char e = '\\''; // gone\n"
           'const char* t = "a \\" // b";\n')
    out = bench.code_of(src)
    assert '"http://x /* y */"' in out
    assert "'\"'" in out and "'\\''" in out
    assert '"a \\" // b"' in out
    assert "gone" not in out


def test_comment_edits_keep_the_code_and_code_edits_change_it():
    base = "x = a + b;  // sum\n/* note */\ny = x * 2;\n"
    reworded = "x = a + b;  // the sum of a and b\n\n// another note\ny = x * 2;\n"
    changed = "x = a - b;  // sum\n/* note */\ny = x * 2;\n"
    assert bench.code_of(base) == bench.code_of(reworded)
    assert bench.code_of(base) != bench.code_of(changed)


def test_source_hash_is_stable_and_covers_the_named_files():
    a = bench.source_sha(bench.DF_SOURCES)
    assert a == bench.source_sha(tuple(reversed(bench.DF_SOURCES)))
    assert len(a) == 16 and int(a, 16) >= 0
    assert a != bench.source_sha(bench.DF_SOURCES[:1])
