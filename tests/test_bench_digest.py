"""bench.py's kernel-source digest (keys the recorded DRAM traffic): it follows
the code and ignores comments and blank space."""
import bench


def test_digest_ignores_comments_and_blank_space():
    a = "int f(int x) {\n  return x + 1;  // one more\n}\n/* block\n comment */\n"
    b = "// header\nint f(int x) {\n\n    return x + 1;\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    files = {"a.cu": a, "b.cu": b, "c.cu": c}
    d = lambda name: bench.src_digest((name,), read=files.__getitem__)  # noqa: E731
    assert d("a.cu") == d("b.cu")
    assert d("a.cu") != d("c.cu")

