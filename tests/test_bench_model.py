"""The benchmark's byte model (the roofline's algorithmic bytes) against the
per-pass accounting of the solve: B(N) = 12 N^2 (N+1) c + 2 N^3 r + (N+1)^3 r
per solve; the field solve P1 + P2 + 3 (P3 + P4 + P5); the non-cubic model
equal to the cubic one on a cube.  No GPU."""
import bench


def test_solve_bytes_sum_to_B():
    for N in (32, 256, 512):
        for c, r in ((8, 4), (16, 8)):
            B = 12 * N * N * (N + 1) * c + 2 * N ** 3 * r + (N + 1) ** 3 * r
            assert sum(bench.pass_bytes(N, c, r)) == B


def test_field_bytes():
    pb = bench.pass_bytes(256, 8, 4)
    assert bench.field_bytes(256, 8, 4) == pb[0] + pb[1] + 3 * (pb[2] + pb[3] + pb[4])


def test_noncubic_model_on_a_cube():
    for N in (16, 64):
        assert bench.pass_bytes3((N, N, N), 8, 4) == bench.pass_bytes(N, 8, 4)
    # the 1 x 1 x 2 box has twice the points and one more spectrum plane per z
    a = bench.pass_bytes3((32, 32, 64), 8, 4)
    assert a[0] == 32 * 32 * 64 * 4 + 64 * 32 * 33 * 8


def test_kernel_source_hash_is_stable():
    assert bench.kernel_src_sha() == bench.kernel_src_sha()
    assert len(bench.kernel_src_sha()) == 16
