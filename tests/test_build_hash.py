"""The hash that ties the recorded DRAM traffic to the step kernel's code
ignores comments and layout but not code."""
from paper_2303_14119_gb300 import _build


def test_code_only_drops_comments_and_layout():
    a = 'int x = 1;  // one\n/* block\n comment */ float y = 2.f;\n'
    b = 'int x = 1;\nfloat y = 2.f; // two'
    assert _build.code_only(a) == _build.code_only(b) == "int x = 1; float y = 2.f;"


def test_code_only_keeps_literals_and_code():
    src = 'asm("mov.u32 %0, 1; // not a comment" : "=r"(v)); char c = \'/\';'
    assert _build.code_only(src) == src
    assert _build.code_only("a = b / c;") != _build.code_only("a = b * c;")
    assert _build.code_only('s = "x\\"//y";') == 's = "x\\"//y";'


def test_source_hash_follows_code(tmp_path):
    f = tmp_path / "k.cu"
    f.write_text("__global__ void k() { int i = 0; }\n")
    h0 = _build.source_hash((str(f),))
    f.write_text("// comment\n__global__ void k() {\n  int i = 0;  // zero\n}\n")
    assert _build.source_hash((str(f),)) == h0
    f.write_text("__global__ void k() { int i = 1; }\n")
    assert _build.source_hash((str(f),)) != h0
