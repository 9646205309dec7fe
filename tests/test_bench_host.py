"""Host-side logic of bench.py."""

def test_traffic_key_ignores_comments_only():
    """bench.py keys the recorded ncu traffic by the kernel code without
    comments: a comment edit keeps the key, a code edit changes it."""
    import bench
    src = "int f(int a) { // add one\n  return a + 1; /* done */ }\n"
    assert bench.code_text(src) == bench.code_text("int f(int a) {\n return a + 1;  }  // changed note\n")
    assert bench.code_text(src) != bench.code_text("int f(int a) { return a + 2; }")
    assert len(bench.source_hash()) == 12
