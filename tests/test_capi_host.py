"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports every symbol
include/lsm.h declares, and its host logic (window schedule, argument validation, status strings)
behaves as documented.  No kernel is launched here."""

import os
import re
import shutil

import numpy as np
import pytest

from oracle import lsm_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1801_00819_gb300 import build as B
    B.build()
    from paper_1801_00819_gb300 import lsm
    return lsm


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "lsm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"typedef[^;]*;", "", src)  # function-pointer types are not entry points
    return sorted(set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src)) - {"if", "sizeof"})


def test_header_declares_expected_entry_points():
    assert _declared_functions() == sorted(["lsm_workspace_bytes", "lsm_forward", "lsm_adjoint", "lsm_num_windows",
                                            "rls_window_solve", "lsm_status_string", "lsm_kernel_launches",
                                            "lsm_profile_start", "lsm_profile_stop", "lsm_adjoint_static",
                                            "lsm_born_gradient", "rls_window_solve_ex", "rls_multi_line_solve",
                                            "lsm_forward_ex", "lsm_adjoint_ex", "lsm_profile_start_classes",
                                            "lsm_autotune", "lsm_autotune_reset", "lsm_autotune_gradient",
                                            "lsm_measure_fp32_peak", "lsm_check_bounded_wait",
                                            "rls_window_solve_sharded", "lsm_fft_tiles", "lsm_set_fft_tile",
                                            "lsm_tcgen05_shape"])


def test_library_exports_every_declared_symbol(lib):
    handle = lib.load_library()
    for name in _declared_functions():
        assert hasattr(handle, name), name
    assert set(lib.EXPORTED) == set(_declared_functions())


def test_window_count_matches_oracle_schedule(lib):
    for ns in range(1, 30):
        for K in range(1, ns + 1):
            for slide in range(1, 7):
                assert lib.lsm_num_windows(ns, K, slide) == len(O.window_starts(ns, K, slide))
    assert lib.lsm_num_windows(240, 5, 3) == 80
    assert lib.lsm_num_windows(5, 6, 1) == 0
    assert lib.lsm_num_windows(5, 2, 0) == 0


def test_profile_without_launches_is_empty(lib):
    lib.lsm_profile_start()
    prof = lib.lsm_profile_stop()
    assert set(prof) == set(lib.KERNEL_CLASSES)
    assert all(v["launches"] == 0 and v["ms"] == 0.0 for v in prof.values())


def test_status_strings(lib):
    assert lib.lsm_status_string(0) == "ok"
    assert "nx" in lib.lsm_status_string(lib.LSM_ERR_UNSUPPORTED_NX)
    assert "896" in lib.lsm_status_string(lib.LSM_ERR_UNSUPPORTED_NX)
    assert lib.lsm_status_string(-99) == "unknown status"


def _holders(lib, nx=64, nz=8, ns=3, nw=4, src=None, rec=None):
    g = lib.Grid(nx, nz, 10.0, 10.0)
    geo = lib.Geometry(np.arange(ns) if src is None else src, rec, nx=nx)
    f = lib.Frequencies(np.linspace(5, 30, nw), np.ones(nw))
    return g, geo, f


def test_validation_rejects_bad_arguments_before_any_launch(lib):
    before = lib.lsm_kernel_launches()
    g, geo, f = _holders(lib)
    fake = 1 << 20  # aligned fake addresses: validation must fail before they are used
    cases = [
        (_holders(lib, nx=40), lib.LSM_ERR_UNSUPPORTED_NX),
        (_holders(lib, nx=1536), lib.LSM_ERR_UNSUPPORTED_NX),
        (_holders(lib, nx=2048), lib.LSM_ERR_UNSUPPORTED_NX),
        (_holders(lib, src=np.array([0, 1, 64])), lib.LSM_ERR_ARG),
        (_holders(lib, rec=np.full((3, 5), 70)), lib.LSM_ERR_ARG),
    ]
    for (gg, gg_geo, gg_f), code in cases:
        with pytest.raises(lib.LsmError) as ei:
            lib.lsm_forward(gg, fake, gg_f, gg_geo, fake, fake, 0, 1, None, stream=0)
        assert ei.value.status == code
    # misaligned device pointer
    with pytest.raises(lib.LsmError) as ei:
        lib.lsm_adjoint(g, fake + 4, f, geo, fake, fake, 0, 1, None, stream=0)
    assert ei.value.status == lib.LSM_ERR_ARG
    # shot range
    with pytest.raises(lib.LsmError):
        lib.lsm_forward(g, fake, f, geo, fake, fake, 2, 2, None, stream=0)
    # window arguments
    with pytest.raises(lib.LsmError):
        lib.rls_window_solve(g, fake, f, geo, fake, -1.0, 2, 1, 0.0, 3, fake, None, stream=0)
    with pytest.raises(lib.LsmError):
        lib.rls_window_solve(g, fake, f, geo, fake, 1.0, 4, 1, 0.0, 3, fake, None, stream=0)
    assert lib.lsm_kernel_launches() == before


def test_static_scratch_variant_rejects_oversize_problems_before_launch(lib):
    before = lib.lsm_kernel_launches()
    g = lib.Grid(512, 256, 8.0, 8.0)
    geo = lib.Geometry(np.arange(16) * 32, None, nx=512)
    f = lib.Frequencies(np.linspace(3, 40, 128), np.ones(128))
    assert lib.lsm_workspace_bytes(g, geo, f, 16, lib.LSM_OP_ADJOINT) > lib.LSM_STATIC_SCRATCH_BYTES
    fake = 1 << 20
    with pytest.raises(lib.LsmError) as ei:
        lib.lsm_adjoint_static(g, fake, f, geo, fake, fake, 0, 16, stream=0)
    assert ei.value.status == lib.LSM_ERR_WORKSPACE
    assert lib.lsm_kernel_launches() == before


def test_fft_tiles_of_every_width(lib):
    """Every width has its default tile and, except 768, 896 and 1024, one with half the points per
    thread (at most 32 threads per item, a multiple of the odd factor)."""
    for nx in (16, 32, 64, 128, 256, 512, 1024, 48, 96, 192, 384, 768, 80, 160, 320, 640, 112, 224, 448, 896):
        tiles = lib.lsm_fft_tiles(nx)
        assert tiles[0] == (32 if nx in (512, 1024) else tiles[0])
        if nx in (768, 896, 1024):
            assert len(tiles) == 1
        else:
            assert len(tiles) == 2 and tiles[1] * 2 == tiles[0] and nx // tiles[1] <= 32
    assert lib.lsm_fft_tiles(40) == []
    with pytest.raises(lib.LsmError):
        lib.lsm_set_fft_tile(512, 16, 128, 8)   # no such tile at 512
    lib.lsm_set_fft_tile(512, 16, 128, 16)
    lib.lsm_autotune_reset()


def test_tensor_core_transform_validation(lib):
    before = lib.lsm_kernel_launches()
    fake = 1 << 20
    g, geo, f = _holders(lib, nx=128, rec=np.tile(np.arange(64), (3, 1)))
    with pytest.raises(lib.LsmError) as ei:  # receiver lists are not taken by the variants
        lib.lsm_adjoint(g, fake, f, geo, fake, fake, 0, 1, None, stream=0, transform="dft_fp16x3")
    assert ei.value.status == lib.LSM_ERR_ARG
    with pytest.raises(ValueError):
        lib._options(transform="fp8")
    assert lib.lsm_kernel_launches() == before


def test_workspace_query_and_too_small_workspace(lib):
    g, geo, f = _holders(lib)
    fwd = lib.lsm_workspace_bytes(g, geo, f, 3, lib.LSM_OP_FORWARD)
    adj = lib.lsm_workspace_bytes(g, geo, f, 3, lib.LSM_OP_ADJOINT)
    sol = lib.lsm_workspace_bytes(g, geo, f, 2, lib.LSM_OP_SOLVE)
    assert 0 < fwd < adj
    # tables (2 x nw nz nx complex) plus the source-wavefield ring dominate
    assert fwd >= (2 + 3) * 4 * 8 * 64 * 8
    assert sol > 0
    assert lib.lsm_workspace_bytes(g, geo, f, 4, lib.LSM_OP_FORWARD) == 0
    assert lib.lsm_workspace_bytes(g, geo, f, 1, 7) == 0

    class FakeWs:
        def __init__(self, n):
            self.n = n

        def numel(self):
            return self.n

        def element_size(self):
            return 1

        def data_ptr(self):
            return 1 << 20
    fake = 1 << 20
    with pytest.raises(lib.LsmError) as ei:
        lib.lsm_forward(g, fake, f, geo, fake, fake, 0, 3, FakeWs(fwd - 1), stream=0)
    assert ei.value.status == lib.LSM_ERR_WORKSPACE


def test_autotune_validation_before_any_launch(lib):
    """lsm_autotune checks its shot count, workspace size and transform on the host first."""
    before = lib.lsm_kernel_launches()
    g, geo, f = _holders(lib)
    sol = lib.lsm_workspace_bytes(g, geo, f, 2, lib.LSM_OP_SOLVE)

    class FakeWs:
        def __init__(self, n):
            self.n = n

        def numel(self):
            return self.n

        def element_size(self):
            return 1

        def data_ptr(self):
            return 1 << 20
    fake = 1 << 20
    for nshots in (0, 4):  # the survey has 3 shots
        with pytest.raises(lib.LsmError) as ei:
            lib.lsm_autotune(g, fake, f, geo, nshots, FakeWs(1 << 30), stream=0)
        assert ei.value.status == lib.LSM_ERR_ARG
    with pytest.raises(lib.LsmError) as ei:
        lib.lsm_autotune(g, fake, f, geo, 2, FakeWs(sol - 1), stream=0)
    assert ei.value.status == lib.LSM_ERR_WORKSPACE
    g2, geo2, f2 = _holders(lib, nx=64, rec=np.tile(np.arange(32), (3, 1)))
    sol2 = lib.lsm_workspace_bytes(g2, geo2, f2, 2, lib.LSM_OP_SOLVE)
    with pytest.raises(lib.LsmError) as ei:  # the tensor-core variants take no receiver list
        lib.lsm_autotune(g2, fake, f2, geo2, 2, FakeWs(sol2), stream=0, transform="dft_bf16x3")
    assert ei.value.status == lib.LSM_ERR_ARG
    lib.lsm_autotune_reset()
    assert lib.lsm_kernel_launches() == before


def test_gradient_stride_tuning_validation_before_any_launch(lib):
    """lsm_autotune_gradient checks its shot count and workspace size on the host first, and the
    gradient workspace reserves room for every candidate stride."""
    before = lib.lsm_kernel_launches()
    g, geo, f = _holders(lib)
    grad = lib.lsm_workspace_bytes(g, geo, f, 2, lib.LSM_OP_GRADIENT)
    assert grad > 0

    class FakeWs:
        def __init__(self, n):
            self.n = n

        def numel(self):
            return self.n

        def element_size(self):
            return 1

        def data_ptr(self):
            return 1 << 20
    fake = 1 << 20
    for nshots in (0, 4):  # the survey has 3 shots
        with pytest.raises(lib.LsmError) as ei:
            lib.lsm_autotune_gradient(g, fake, f, geo, nshots, FakeWs(1 << 30), stream=0)
        assert ei.value.status == lib.LSM_ERR_ARG
    with pytest.raises(lib.LsmError) as ei:
        lib.lsm_autotune_gradient(g, fake, f, geo, 2, FakeWs(grad - 1), stream=0)
    assert ei.value.status == lib.LSM_ERR_WORKSPACE
    lib.lsm_autotune_reset()
    assert lib.lsm_kernel_launches() == before


def test_tcgen05_launch_shapes(lib):
    """The tcgen05 variants' launch shape per width (host only): items and threads per CTA, CTAs,
    and the fall-back to unstaged Phi and D rows when a CTA's frequencies would not fit its shared
    memory (nx = 1024 windows of one or two shots)."""
    for nx, items, threads in ((128, 16, 128), (256, 8, 128), (512, 8, 128), (1024, 8, 256)):
        sh = lib.lsm_tcgen05_shape(nx, 16, 128)
        assert (sh["items"], sh["threads"]) == (items, threads)
        assert sh["blocks"] == (16 * 128 + items - 1) // items and sh["wslots"] == 2
        assert sh["smem_bytes"] <= 227 * 1024 - 1024
    assert lib.lsm_tcgen05_shape(1024, 3, 10)["wslots"] == 4
    assert lib.lsm_tcgen05_shape(1024, 2, 10)["wslots"] == 0
    assert lib.lsm_tcgen05_shape(1024, 1, 10)["wslots"] == 0
    assert lib.lsm_tcgen05_shape(512, 1, 10)["wslots"] == 9
    assert lib.lsm_tcgen05_shape(128, 1, 40)["wslots"] == 17
    assert lib.lsm_tcgen05_shape(512, 2, 3)["wslots"] == 3  # at most nw
    for nx in (64, 384, 2048):
        with pytest.raises(lib.LsmError) as ei:
            lib.lsm_tcgen05_shape(nx, 4, 4)
        assert ei.value.status == lib.LSM_ERR_UNSUPPORTED_NX
    with pytest.raises(lib.LsmError):
        lib.lsm_tcgen05_shape(512, 0, 4)


def test_header_constants_match_binding(lib):
    """Every integer #define LSM_* of include/lsm.h that the binding mirrors has the header's value,
    and the status, op, transform and graph-mode codes are all mirrored."""
    src = open(os.path.join(ROOT, "include", "lsm.h")).read()
    defs = {m.group(1): int(m.group(2))
            for m in re.finditer(r"#define\s+(LSM_[A-Z0-9_]+)\s+\(?(-?\d+)\)?(?=\s|$)", src, flags=re.M)}
    assert defs, "no constants parsed"
    assert "(64u << 20)" in src and lib.LSM_STATIC_SCRATCH_BYTES == 64 << 20
    for name, value in defs.items():
        if hasattr(lib, name):
            assert getattr(lib, name) == value, name
    for prefix in ("LSM_ERR_", "LSM_OP_", "LSM_CUDA_GRAPH_"):
        for name in (n for n in defs if n.startswith(prefix)):
            assert hasattr(lib, name), name
