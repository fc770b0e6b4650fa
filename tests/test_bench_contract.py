"""The benchmark's bookkeeping, on the CPU: the algorithmic bytes behind the
roofline fractions and the recorded ncu traffic entries."""
import bench

N_SITES = 216_576 + 72_192  # water72192: atoms + Wannier centroids


def test_algorithmic_bytes_per_kernel_128():
    """Closed forms at 128^3 (FP32): N = 2,097,152 mesh points, N_h =
    128 x 128 x 65 half-spectrum points, n = 288,768 sites."""
    a = bench.algorithmic_bytes(N_SITES, 128)
    N, NH, n = 128 ** 3, 128 * 128 * 65, N_SITES
    assert a["spread"] == 16 * n + 4 * N == 13_008_896
    assert a["gather"] == 12 * N + 28 * n == 33_251_328
    assert a["fft_x_influence"] == 28 * NH == 29_818_880
    assert a["fft_y_inverse3"] == 40 * NH
    assert a["fft_z_c2r"] == 24 * NH + 12 * N
    assert a["scan"] == 0


def test_step_bytes_are_the_method_minimum():
    """One forward pass over the mesh and three inverse ones, the influence,
    the spread and the gather: 126.7 MB at 128^3, 235.0 MB at 160^3."""
    assert bench.step_algorithmic_bytes(N_SITES, 128) == 126_672_896
    assert bench.step_algorithmic_bytes(N_SITES, 160) == 235_016_192
    a = bench.algorithmic_bytes(N_SITES, 128)
    # the per-kernel figures of the passes the step is made of add up to it
    # except where a pass reads or writes more than the minimum (the y passes)
    parts = a["spread"] + a["fft_z_r2c"] + a["gather"]
    assert parts < bench.step_algorithmic_bytes(N_SITES, 128)


def test_recorded_traffic_names_real_kernels():
    names = set(bench.algorithmic_bytes(N_SITES, 128))
    for (kernel, mesh), traffic in bench.NCU_TRAFFIC.items():
        assert kernel in names and mesh in (128, 160)
        # cold-L2 DRAM bytes of one launch: at least the compulsory reads of
        # the sites or mesh, at most a few times the algorithmic bytes
        alg = bench.algorithmic_bytes(N_SITES, mesh)[kernel]
        assert 0.2 * alg < traffic < 4 * alg, (kernel, mesh, traffic, alg)


def test_oracle_pool_on_host_cores():
    """The CPU baseline's process pool (spawned workers, one thread each)
    evaluates the frames it is given: two workers, one timed round on the
    64-water box."""
    from workloads.water import make_workload
    wb, w = make_workload("water64")
    val, rates, workers = bench.oracle_all_cores(wb, w, lambda k: wb.pos + 0.01 * k, rounds=1, workers=2)
    assert workers == 2 and len(rates) == 1 and val > 0
