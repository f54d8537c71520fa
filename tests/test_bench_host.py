"""Host-side logic of the benchmark that needs no GPU: the digest that ties a
committed ncu summary to the kernel code it was taken on."""
import bench

CODE = """// pass over a chunk
__device__ float f(float x) {   /* one
  FMA */ return fmaf(x, x, 1.0f);  // trailing note
}
"""


def test_digest_ignores_comments_and_blank_lines():
    edited = CODE.replace("// pass over a chunk", "// a reworded comment\n\n") \
                 .replace("/* one\n  FMA */", "/* another */")
    assert bench.code_digest([CODE]) == bench.code_digest([edited])


def test_digest_follows_the_code():
    assert bench.code_digest([CODE]) != bench.code_digest([CODE.replace("1.0f", "2.0f")])
    # the order of the files is part of the digest
    other = "__global__ void k() {}\n"
    assert bench.code_digest([CODE, other]) != bench.code_digest([other, CODE])

