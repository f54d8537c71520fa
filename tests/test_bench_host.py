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



def test_pass_roofline_splits_floor_and_decaying_iterations():
    """Fractions from per-iteration device timestamps: a pass's algorithmic
    FP32 instructions over its time, against the peak; iterations at the
    smallest lengthscale are the floor, the others decaying."""
    wpp = {"grad": 22, "step": 52, "mufu": 1}
    rec = dict(plan_ms=0.0, grad_ms=0.0, step_ms=0.0, grad_sync_ms=0.0, step_sync_ms=0.0,
               grad_pairs=0, step_pairs=0)
    a = dict(rec, ell=0.15, plan_ms=0.01, grad_ms=0.05, step_ms=0.07, grad_sync_ms=0.04,
             step_sync_ms=0.05, grad_pairs=10_000_000, step_pairs=10_000_000)
    b = dict(rec, ell=0.02, grad_ms=0.01, step_ms=0.02, grad_sync_ms=0.008, step_sync_ms=0.012,
             grad_pairs=1_000_000, step_pairs=1_000_000)
    out = bench.pass_roofline([a, b, b], wpp, peak_fp32=40.0)
    assert out["floor"]["iters"] == 2 and out["decaying"]["iters"] == 1
    g = out["decaying"]["gradient"]
    # 1e7 pairs x 22 inst in 40 us = 5.5 T inst/s of a 40 T peak
    assert abs(g["frac"] - 5.5 / 40.0) < 1e-12
    st = out["floor"]["step"]
    assert st["pairs"] == 2_000_000 and abs(st["pass_ms"] - 0.024) < 1e-15
    assert abs(st["frac"] - 2e6 * 52 / 24e-6 / 1e12 / 40.0) < 1e-12
    it = out["all"]["iteration"]
    assert abs(it["ms"] - (0.13 + 2 * 0.03)) < 1e-12
    assert abs(it["tails_ms"] - (it["ms"] - it["plan_ms"] - out["all"]["both_passes"]["pass_ms"])) < 1e-15
    assert bench.pass_roofline([], wpp, 40.0) is None
