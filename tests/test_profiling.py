"""Host-side checks of the ncu summary helpers (no GPU)."""
from paper_2602_01723_gb300.profiling import source_hash, strip_comments


def test_comments_are_stripped_and_literals_kept():
    src = 'int a = 1; // one\nconst char *s = "x // y /* z */"; /* two\nlines */ char q = \'"\'; int b = a / 2;\n'
    out = strip_comments(src)
    assert "one" not in out and "two" not in out and "lines" not in out
    assert '"x // y /* z */"' in out and "'\"'" in out and "a / 2" in out


def test_escaped_quotes_do_not_end_a_literal():
    out = strip_comments('const char *s = "a\\" // b"; int c; // d\n')
    assert '"a\\" // b"' in out and "int c;" in out and "d" not in out.split("int c;")[1]


def test_hash_is_stable():
    assert source_hash() == source_hash() and len(source_hash()) == 16
