"""CPU-side checks of the C ABI: the library loads, exports every function
include/fastergs.h declares, its structs match the ctypes mirrors, and the
host-only logic (workspace layout, argument checks, status strings) behaves.
No call here launches a kernel."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2602_09999_gb300 import binding as B
from paper_2602_09999_gb300 import build_lib, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastergs.h")


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return B.lib()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fgs_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(B.EXPORTED)


def test_struct_sizes_match_c(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "fastergs.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(fgs_camera),'
                   ' sizeof(fgs_params), sizeof(fgs_workspace_layout), sizeof(fgs_adam_state),'
                   ' offsetof(fgs_adam_state, step_size), offsetof(fgs_workspace_layout, tuning),'
                   ' offsetof(fgs_tuning, backward_pixels_per_thread), offsetof(fgs_tuning, backward_batch),'
                   ' offsetof(fgs_tuning, duplicate_order));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(x) for x in out] == [ctypes.sizeof(B.fgs_camera), ctypes.sizeof(B.fgs_params),
                                     ctypes.sizeof(B.fgs_workspace_layout),
                                     ctypes.sizeof(B.fgs_adam_state),
                                     B.fgs_adam_state.step_size.offset,
                                     B.fgs_workspace_layout.tuning.offset,
                                     B.fgs_tuning.backward_pixels_per_thread.offset,
                                     B.fgs_tuning.backward_batch.offset,
                                     B.fgs_tuning.duplicate_order.offset]


def test_workspace_layout(lib):
    cams = [scenes.look_at((0, 0, 4), (0, 0, 0), w, h) for w, h in [(1237, 822), (640, 426)]]
    ca = B.camera_array(cams)
    L = B.fgs_workspace_size(3_000_000, ca, 2, 10_000_000)
    tiles = 78 * 52 + 40 * 27
    assert L.total_tiles == tiles
    assert L.total_pixels == 1237 * 822 + 640 * 426
    assert L.sort_bits == int(np.ceil(np.log2(tiles)))
    assert L.sorted_in_alt == ((L.sort_bits + 7) // 8) % 2
    offs = list(L.offset)
    sizes = list(L.bytes)
    for i in range(B.FGS_WS_NUM_SLOTS):
        assert offs[i] % 256 == 0
        if i + 1 < B.FGS_WS_NUM_SLOTS:
            assert offs[i] + sizes[i] <= offs[i + 1]
    assert offs[-1] + sizes[-1] <= L.total_bytes
    assert sizes[B.FGS_WS_SCREEN] == 48 * 2 * 3_000_000
    assert sizes[B.FGS_WS_KEYS] == 4 * 10_000_000
    assert sizes[B.FGS_WS_DEPTH_KEYS] == 4 * 2 * 3_000_000


@pytest.mark.parametrize("n,nv,k,code", [(0, 1, 10, -2), (2 ** 31, 1, 10, -2), (10, 0, 10, -7),
                                         (10, 17, 10, -7), (10, 1, -1, -9),
                                         # view * n + index must fit the 32-bit pair value
                                         (2 ** 28, 16, 10, -2)])
def test_workspace_argument_errors(lib, n, nv, k, code):
    cams = [scenes.look_at((0, 0, 4), (0, 0, 0), 64, 64)] * max(nv, 1)
    ca = B.camera_array(cams)
    with pytest.raises(B.FGSError) as e:
        B.fgs_workspace_size(n, ca, nv, k)
    assert e.value.code == code


def test_largest_pair_count_accepted(lib):
    # n_views * n = 2^32 - 16: the layout is host arithmetic, nothing is allocated
    cams = [scenes.look_at((0, 0, 4), (0, 0, 0), 64, 64)] * 16
    L = B.fgs_workspace_size(2 ** 28 - 1, B.camera_array(cams), 16, 10)
    assert L.bytes[B.FGS_WS_DEPTH_KEYS] == 4 * 16 * (2 ** 28 - 1)


def test_bad_camera_size_rejected(lib):
    cam = scenes.look_at((0, 0, 4), (0, 0, 0), 64, 64)
    cam.width = 0
    with pytest.raises(B.FGSError) as e:
        B.fgs_workspace_size(10, B.camera_array([cam]), 1, 10)
    assert e.value.code == -2


def test_strerror(lib):
    for code in range(-10, 1):
        assert B.fgs_strerror(code) != "unknown status"
    assert B.fgs_strerror(-100) == "unknown status"


def _header_enum(name):
    """{member: value} of one enum of the header, read as text."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"enum\s+" + name + r"\s*\{(.*?)\}", text, flags=re.S).group(1)
    out = {}
    for item in body.split(","):
        m = re.match(r"\s*(\w+)\s*=\s*(-?\w+)", item)
        if m:
            out[m.group(1)] = int(m.group(2).rstrip("uU"), 0)
    return out


def test_device_flags_and_their_strings(lib):
    """The sticky device flags: distinct single bits, mirrored by the
    binding, each with its own description; anything else is unknown."""
    flags = _header_enum("fgs_device_flags")
    assert flags == {"FGS_FLAG_CAPACITY": B.FGS_FLAG_CAPACITY,
                     "FGS_FLAG_NONFINITE": B.FGS_FLAG_NONFINITE}
    bits = list(flags.values())
    assert all(b and (b & (b - 1)) == 0 for b in bits) and len(set(bits)) == len(bits)
    texts = {B.fgs_flag_string(b) for b in bits}
    assert len(texts) == len(bits) and "unknown flag" not in texts
    assert "NaN" in B.fgs_flag_string(B.FGS_FLAG_NONFINITE)
    for other in (0, 4, B.FGS_FLAG_CAPACITY | B.FGS_FLAG_NONFINITE, 0xffffffff):
        assert B.fgs_flag_string(other) == "unknown flag"
    assert _header_enum("fgs_status") == {v: k for k, v in B.STATUS.items()}


def test_null_pointer_checks_before_any_launch(lib):
    """Argument checks run on the host before any CUDA call."""
    cam = B.camera_array([scenes.look_at((0, 0, 4), (0, 0, 0), 64, 64)])
    L = B.fgs_workspace_size(10, cam, 1, 100)
    with pytest.raises(B.FGSError) as e:
        B.fgs_render_forward(None, L, B.fgs_params(), 3, cam, None, (0, 0, 0), None, None)
    assert e.value.code == -1
    with pytest.raises(B.FGSError) as e:
        B.fgs_adam_step(B.fgs_params(), B.fgs_params(), B.fgs_params(), B.fgs_params(),
                        [1e-3] * 6, 0.9, 0.999, 1e-15, 1, None)
    assert e.value.code in (-1, -2)
    with pytest.raises(B.FGSError) as e:
        B.fgs_sort_pairs(None, None, None, None, 10, 32, None, 0, None)
    assert e.value.code == -1
    with pytest.raises(B.FGSError) as e:
        B.fgs_render_backward_adam(None, L, B.fgs_params(), 3, cam, None, (0, 0, 0), None,
                                   B.fgs_params(), B.fgs_params(), None, None, None)
    assert e.value.code == -1


def test_sort_alignment_checks_before_any_launch(lib):
    """Misaligned key (8-byte) or value (4-byte) buffers are rejected on the
    host; the fake addresses are never dereferenced."""
    base = 1 << 40
    sb = B.fgs_sort_scratch_bytes(10)
    good = dict(keys=base, vals=base + (1 << 32), keys_alt=base + (2 << 32), vals_alt=base + (3 << 32))
    for name, off in (("keys", 4), ("vals", 2), ("keys_alt", 4), ("vals_alt", 1)):
        a = dict(good)
        a[name] += off
        with pytest.raises(B.FGSError) as e:
            B.fgs_sort_pairs(a["keys"], a["vals"], a["keys_alt"], a["vals_alt"], 10, 32,
                             base + (4 << 32), sb, None)
        assert e.value.code == -8, name
    for k, v in ((base + 4, base + (1 << 32)), (base, base + (1 << 32) + 2)):
        with pytest.raises(B.FGSError) as e:
            B.fgs_sort_pairs_static(k, v, 10, 32, None)
        assert e.value.code == -8


def _fake_params(n, base, dtypes=None, groups=6):
    """fgs_params over fake, never dereferenced device addresses."""
    ptrs = [base + (g << 32) for g in range(groups)]
    return B.params_struct(n, ptrs, dtypes or [B.FGS_F32] * groups)


def test_morton_and_permute_argument_checks(lib):
    """Host checks of the z-order entry points, before any CUDA call."""
    P = ctypes.c_void_p
    sb = B.fgs_morton_scratch_bytes(1000)
    assert sb >= 3 * 4 * 1000
    assert lib.fgs_morton_order(None, 0, None, None, None, 0, None) == 0      # n = 0: no-op
    assert lib.fgs_morton_order(None, -1, None, None, None, 0, None) == -2
    assert lib.fgs_morton_order(None, 1000, None, None, None, sb, None) == -1
    assert lib.fgs_morton_order(P(4096), 1000, P(8192), None, P(1 << 20), sb - 1, None) == -4
    assert lib.fgs_morton_order(P(4096), 1000, P(8192), None, P((1 << 20) + 16), sb, None) == -8
    src = _fake_params(10, 1 << 40)
    dst = _fake_params(10, 1 << 44)
    with pytest.raises(B.FGSError) as e:
        B.fgs_permute_params(B.params_struct(10, [0] * 6, [B.FGS_F32] * 6), dst, None, None)
    assert e.value.code == -1
    bad = _fake_params(10, 1 << 44, [B.FGS_F32] * 4 + [B.FGS_BF16] * 2)
    with pytest.raises(B.FGSError) as e:                      # storage types differ
        B.fgs_permute_params(src, bad, None, None)
    assert e.value.code == -5
    with pytest.raises(B.FGSError) as e:                      # dst overlaps src
        B.fgs_permute_params(src, src, None, None)
    assert e.value.code == -9
    extra = _fake_params(10, 1 << 44, [B.FGS_F32] * 8, groups=8)
    with pytest.raises(B.FGSError) as e:                      # dst has groups src lacks
        B.fgs_permute_params(src, extra, None, None)
    assert e.value.code == -9
    short = _fake_params(9, 1 << 44)
    with pytest.raises(B.FGSError) as e:
        B.fgs_permute_params(src, short, None, None)
    assert e.value.code == -2
    empty_src, empty_dst = _fake_params(0, 1 << 40), _fake_params(0, 1 << 44)
    B.fgs_permute_params(empty_src, empty_dst, None, None)    # n = 0: no-op


def test_per_gaussian_layout_and_checks(lib):
    """The per-Gaussian buffers exist only with FGS_WS_PER_GAUSSIAN, sized
    by k_max and the tile count; selecting that backward on a layout made
    without them, or an unknown backward, is rejected before any launch."""
    cam = B.camera_array([scenes.look_at((0, 0, 4), (0, 0, 0), 100, 70)])
    plain = B.fgs_workspace_size(1000, cam, 1, 64_000)
    pg = B.fgs_workspace_size_ex(1000, cam, 1, 64_000, B.FGS_WS_PER_GAUSSIAN)
    tiles = 7 * 5
    for s in (B.FGS_WS_BUCKET_OFF, B.FGS_WS_BUCKET_TILE, B.FGS_WS_BUCKET_STATE, B.FGS_WS_PIXEL_FINAL):
        assert plain.bytes[s] == 0
    assert pg.bytes[B.FGS_WS_BUCKET_OFF] == 4 * (tiles + 1)
    assert pg.bytes[B.FGS_WS_BUCKET_TILE] == 4 * (64_000 // 32 + tiles)
    assert pg.bytes[B.FGS_WS_BUCKET_STATE] == 16 * 256 * (64_000 // 32 + tiles)
    assert pg.bytes[B.FGS_WS_PIXEL_FINAL] == 16 * 100 * 70
    assert pg.flags == B.FGS_WS_PER_GAUSSIAN and plain.flags == 0
    assert pg.tuning.blend_backward == B.FGS_BACKWARD_PER_PIXEL
    with pytest.raises(B.FGSError) as e:
        B.fgs_workspace_size_ex(1000, cam, 1, 64_000, 2)
    assert e.value.code == -9
    fake_ws = ctypes.c_void_p(1 << 20)
    p = B.params_struct(1000, [1 << 40] * 6, [B.FGS_F32] * 6)
    plain.tuning.blend_backward = B.FGS_BACKWARD_PER_GAUSSIAN
    with pytest.raises(B.FGSError) as e:
        B.fgs_render_forward(fake_ws, plain, p, 3, cam, 1 << 30, (0, 0, 0), 1 << 31, None)
    assert e.value.code == -4
    pg.tuning.blend_backward = 7
    with pytest.raises(B.FGSError) as e:
        B.fgs_render_forward(fake_ws, pg, p, 3, cam, 1 << 30, (0, 0, 0), 1 << 31, None)
    assert e.value.code == -9
    # the backward's own launch pair: (0, 0) by default, else a supported pair
    pg.tuning.blend_backward = B.FGS_BACKWARD_PER_PIXEL
    assert (pg.tuning.backward_pixels_per_thread, pg.tuning.backward_batch) == (0, 0)
    for pair in ((4, 32), (0, 128), (3, 128)):
        pg.tuning.backward_pixels_per_thread, pg.tuning.backward_batch = pair
        with pytest.raises(B.FGSError) as e:
            B.fgs_render_forward(fake_ws, pg, p, 3, cam, 1 << 30, (0, 0, 0), 1 << 31, None)
        assert e.value.code == -9, pair


def test_misaligned_quaternions_rejected(lib):
    """Quaternion rows are read as one 16-byte vector: a buffer off a
    16-byte boundary is FGS_ERR_ALIGN before any launch."""
    cam = B.camera_array([scenes.look_at((0, 0, 4), (0, 0, 0), 64, 64)])
    L = B.fgs_workspace_size(1000, cam, 1, 64_000)
    ptrs = [1 << 40, 1 << 41, (1 << 42) + 4, 1 << 43, 1 << 44, 1 << 45]
    p = B.params_struct(1000, ptrs, [B.FGS_F32] * 6)
    with pytest.raises(B.FGSError) as e:
        B.fgs_render_forward(ctypes.c_void_p(1 << 20), L, p, 3, cam, 1 << 30, (0, 0, 0), 1 << 31, None)
    assert e.value.code == -8


def test_tuning_choice_encoding(lib):
    """The autotuner's choice tuples map onto the layout's launch fields: a
    backward pair of (0, 0), or none, means the forward's pair; labels name
    every field that is set, so the three tuning passes never share one."""
    from paper_2602_09999_gb300 import tune
    cam = B.camera_array([scenes.tiny_camera(100, 70)])
    layout = B.fgs_workspace_size(1000, cam, 1, 64_000)
    t = layout.tuning
    tune.apply(layout, (4, 64, B.FGS_SCHEDULE_GRID, 2, 256))
    assert (t.blend_pixels_per_thread, t.blend_batch, t.blend_schedule) == (4, 64, B.FGS_SCHEDULE_GRID)
    assert (t.backward_pixels_per_thread, t.backward_batch) == (2, 256)
    tune.apply(layout, (2, 128))
    assert (t.blend_schedule, t.backward_pixels_per_thread, t.backward_batch) == (B.FGS_SCHEDULE_QUEUE, 0, 0)
    assert tune.label((2, 128, 0, 0, 0)) == tune.label((2, 128, 0)) == "2x128/queue"
    assert tune.label((2, 128, 1, 4, 64)) == "2x128/grid+bwd4x64"
    first = [tuple(c) + (0, 0) for c in tune.all_choices()]
    best = (2, 128, 0)
    second = [best + tuple(pb) for pb in B.BLEND_CONFIGS if tuple(pb) != best[:2]]
    third = [tuple(pb) + (0, 4, 64) for pb in B.BLEND_CONFIGS if tuple(pb) != best[:2]]
    sorts = [best + (0, 0, d, t) for d in B.SORT_DIGIT_BITS for t in B.SORT_DIGIT_BITS if (d, t) != (8, 8)]
    dup = [best + (0, 0, 0, 0, B.FGS_DUPLICATE_SPLIT)]
    labels = [tune.label(c) for c in first + second + third + sorts + dup]
    assert len(set(labels)) == len(labels)
    assert tune.label(best + (0, 0, 0, 0, B.FGS_DUPLICATE_STRIDED)) == tune.label(best)


def test_duplicate_order_choice(lib):
    """The duplication order: strided by default, split when the choice's
    eighth field asks for it; any other value is refused on the host."""
    from paper_2602_09999_gb300 import tune
    cam = B.camera_array([scenes.tiny_camera(100, 70)])
    layout = B.fgs_workspace_size(1000, cam, 1, 64_000)
    assert layout.tuning.duplicate_order == B.FGS_DUPLICATE_STRIDED
    tune.apply(layout, (2, 128, 0, 0, 0, 0, 0, B.FGS_DUPLICATE_SPLIT))
    assert layout.tuning.duplicate_order == B.FGS_DUPLICATE_SPLIT
    assert tune.label((2, 128, 0, 0, 0, 0, 0, 1)) == "2x128/queue+dupsplit"
    tune.apply(layout, (2, 128, 0, 0, 0, 8, 8))
    assert layout.tuning.duplicate_order == B.FGS_DUPLICATE_STRIDED
    fake_ws = ctypes.c_void_p(1 << 20)
    p = B.params_struct(1000, [1 << 40] * 6, [B.FGS_F32] * 6)
    for bad in (2, -1):
        layout.tuning.duplicate_order = bad
        with pytest.raises(B.FGSError) as e:
            B.fgs_render_forward(fake_ws, layout, p, 3, cam, 1 << 30, (0, 0, 0), 1 << 31, None)
        assert e.value.code == -9, bad


def test_sort_digit_width_choice(lib):
    """The radix digit widths: 8 or 11 bits (0 means 8) for each sort; the
    tile sort's width decides where its result ends (sorted_in_alt, the
    parity of its pass count), which tune.apply keeps in step and every call
    checks on the host."""
    from paper_2602_09999_gb300 import tune
    cam = B.camera_array([scenes.look_at((0, 0, 4), (0, 0, 0), 1237, 822)])
    layout = B.fgs_workspace_size(1000, cam, 1, 64_000)
    assert layout.sort_bits == 12 and layout.sorted_in_alt == 0          # 8 + 4 bits: two passes
    tune.apply(layout, (2, 128, 0, 0, 0, 11, 11))
    assert (layout.tuning.depth_sort_digit_bits, layout.tuning.tile_sort_digit_bits) == (11, 11)
    assert layout.sorted_in_alt == 0                                      # 11 + 1 bits: two passes
    small = B.fgs_workspace_size(1000, B.camera_array([scenes.tiny_camera(100, 70)]), 1, 64_000)
    assert small.sort_bits == 6 and small.sorted_in_alt == 1              # 35 tiles: one pass
    tune.apply(small, (2, 128, 0, 0, 0, 8, 11))
    assert small.sorted_in_alt == 1
    assert tune.label((2, 128, 0, 0, 0, 11, 0)) == "2x128/queue+sort11/8"
    fake_ws = ctypes.c_void_p(1 << 20)
    p = B.params_struct(1000, [1 << 40] * 6, [B.FGS_F32] * 6)
    for bad in ((9, 8), (8, 16), (-1, 0)):
        layout.tuning.depth_sort_digit_bits, layout.tuning.tile_sort_digit_bits = bad
        with pytest.raises(B.FGSError) as e:
            B.fgs_render_forward(fake_ws, layout, p, 3, cam, 1 << 30, (0, 0, 0), 1 << 31, None)
        assert e.value.code == -9, bad
    # a sorted_in_alt out of step with the tile sort's width
    tune.apply(small, (2, 128, 0, 0, 0, 8, 8))
    small.sorted_in_alt = 0
    scam = B.camera_array([scenes.tiny_camera(100, 70)])
    with pytest.raises(B.FGSError) as e:
        B.fgs_render_forward(fake_ws, small, p, 3, scam, 1 << 30, (0, 0, 0), 1 << 31, None)
    assert e.value.code == -4
