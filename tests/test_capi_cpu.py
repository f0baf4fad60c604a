"""The C-ABI library on a machine without a GPU: it builds and loads, exports
every function include/gmm.h declares, and rejects bad arguments on the host
before touching the device. No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2110_14934_gb300 as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(gmm_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = G.load_library()
    names = declared_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_config_defaults():
    L = G.load_library()
    cfg = G.GMMConfig()
    L.gmm_config_init(ctypes.byref(cfg), 480, 640, 3, 0.01, 2.5, 0.7, 225.0, 0.05)
    assert (cfg.H, cfg.W, cfg.M) == (480, 640, 3)
    assert cfg.init_var_d == np.float32(225.0) and cfg.v_min_c == 1.0 and cfg.v_min_d == 1.0
    assert cfg.precision == G.PREC_F32 and cfg.morph_open == 0
    assert cfg.mode == G.MODE_FUSION and cfg.flags == 0
    assert cfg.depth_scale == np.float32(255.0 / 4095.0)


def test_config_struct_matches_header():
    """The ctypes mirror of gmm_config lists the header's fields in order."""
    text = open(os.path.join(ROOT, "include", "gmm.h")).read()
    body = text[text.index("typedef struct gmm_config {"):text.index("} gmm_config;")]
    names = []
    for decl in re.findall(r"^\s*(?:unsigned\s+)?(?:int|float)\s+([^;]+);", body, re.M):
        names += [n.strip() for n in decl.split(",")]
    assert names == [f[0] for f in G.GMMConfig._fields_]


@pytest.mark.parametrize("args,frag", [
    ((0, 640, 3, 0.01, 2.5, 0.7, 225.0, 0.05), "H and W"),
    ((480, 0, 3, 0.01, 2.5, 0.7, 225.0, 0.05), "H and W"),
    ((480, 640, 2, 0.01, 2.5, 0.7, 225.0, 0.05), "M must be in [3, 5]"),
    ((480, 640, 6, 0.01, 2.5, 0.7, 225.0, 0.05), "M must be in [3, 5]"),
    ((480, 640, 3, 0.0, 2.5, 0.7, 225.0, 0.05), "alpha"),
    ((480, 640, 3, 1.0, 2.5, 0.7, 225.0, 0.05), "alpha"),
    ((480, 640, 3, float("nan"), 2.5, 0.7, 225.0, 0.05), "alpha"),
    ((480, 640, 3, 0.01, 0.0, 0.7, 225.0, 0.05), "match_k"),
    ((480, 640, 3, 0.01, float("inf"), 0.7, 225.0, 0.05), "match_k"),
    ((480, 640, 3, 0.01, 2.5, 1.0, 225.0, 0.05), "bg_T"),
    ((480, 640, 3, 0.01, 2.5, 0.0, 225.0, 0.05), "bg_T"),
    ((480, 640, 3, 0.01, 2.5, 0.7, 0.0, 0.05), "init_var"),
    ((480, 640, 3, 0.01, 2.5, 0.7, 225.0, 0.0), "init_w"),
    ((480, 640, 3, 0.01, 2.5, 0.7, 225.0, 1.0), "init_w"),
    ((1 << 16, 1 << 16, 3, 0.01, 2.5, 0.7, 225.0, 0.05), "too large"),
])
def test_create_rejects_bad_parameters(args, frag):
    L = G.load_library()
    h = L.gmm_create(*args)
    assert not h
    assert frag in L.gmm_last_error().decode()


def test_create_ex_rejects_bad_extensions():
    L = G.load_library()
    cfg = G.GMMConfig()
    L.gmm_config_init(ctypes.byref(cfg), 48, 64, 4, 0.01, 2.5, 0.7, 225.0, 0.05)
    for field, val, frag in (("v_min_c", 0.0, "floors"), ("v_min_d", -1.0, "floors"),
                             ("init_var_d", 0.0, "init_var_d"), ("precision", 7, "precision"),
                             ("morph_open", 2, "morph_open"), ("mode", 2, "mode"),
                             ("depth_scale", 0.0, "depth_scale"),
                             ("depth_scale", float("inf"), "depth_scale"),
                             ("flags", 8, "flags"), ("flags", 4, "needs GMM_PREC_F16")):
        c = G.GMMConfig.from_buffer_copy(cfg)
        setattr(c, field, val)
        assert not L.gmm_create_ex(ctypes.byref(c))
        assert frag in L.gmm_last_error().decode()


def test_null_handles_are_rejected():
    L = G.load_library()
    assert L.gmm_apply(None, None, None, None) == G.EINVAL
    assert L.gmm_state_get(None, 0, 0, None, 0) == G.EINVAL
    assert L.gmm_destroy(None) == G.EINVAL
    assert L.gmm_pool_tick(None) == G.EINVAL
    assert L.gmm_pool_admit(None, None) == G.EINVAL
    assert L.gmm_fuse_masks(None, None, None, None, 4, 4, None) == G.EINVAL
    assert L.gmm_morph_open3(None, None, 0, 4, None) == G.EINVAL
    assert L.gmm_pool_create(0, 3, 4) is None
    assert L.gmm_pool_create(0, 0, 0) is None


def test_sizes():
    assert [G.mask_words_per_row(w) for w in (1, 31, 32, 33, 640, 1920)] == [1, 1, 1, 2, 20, 60]
    # 256-pixel tiles of 8*M planes (4 or 2 bytes each) plus one List-1 byte per tiled pixel
    n = 480 * 640
    assert G.state_bytes(480, 640, 3, G.PREC_F32) == 3 * 8 * n * 4 + n
    assert G.state_bytes(1080, 1920, 5, G.PREC_F16) == 5 * 8 * 1080 * 1920 * 2 + 1080 * 1920
    assert G.state_bytes(1, 1, 3, G.PREC_F32) == 24 * 256 * 4 + 256
    assert G.state_bytes(3, 33, 4, G.PREC_F16) == 32 * 256 * 2 + 256
    assert G.state_bytes(10, 10, 2, G.PREC_F32) == 0


def test_mask_pack_roundtrip():
    rng = np.random.default_rng(0)
    for H, W in ((1, 1), (3, 33), (7, 64), (5, 100)):
        m = rng.random((H, W)) < 0.5
        words = G.pack_mask(m)
        assert words.shape == (H, G.mask_words_per_row(W))
        assert np.array_equal(G.unpack_mask(words, H, W), m)
    # bit i of word c is pixel 32c + i, least significant bit first
    m = np.zeros((1, 40), bool); m[0, 0] = True; m[0, 33] = True
    assert G.pack_mask(m).tolist() == [[1, 2]]


def test_server_host_checks():
    L = G.load_library()
    assert L.gmm_server_create(0, 7, 4, 4) is None
    assert L.gmm_server_create(0, 0, 0, 4) is None
    assert L.gmm_server_create(0, 0, 4, 0) is None
    assert L.gmm_server_admit(None, None) == G.EINVAL
    assert L.gmm_server_push(None, 0, None, None, None, 0.0) == G.EINVAL
    assert L.gmm_server_wait(None, 0, 0) == G.EINVAL
    assert L.gmm_server_destroy(None, 0) == G.EINVAL
    assert L.gmm_server_reserve(None, 0, 0) == G.EINVAL
    assert L.gmm_server_set_transfer(None, G.SERVE_COPY) == G.EINVAL
    assert L.gmm_pool_reserve(None, 0) == G.EINVAL
    t0 = L.gmm_server_now()
    t1 = L.gmm_server_now()
    assert t1 >= t0 > 0


def test_server_trace_struct_matches_header():
    """The ctypes mirror of gmm_server_trace lists the header's fields in
    order, with C's layout (56 bytes, no padding)."""
    text = open(os.path.join(ROOT, "include", "gmm.h")).read()
    body = text[text.index("typedef struct gmm_server_trace {"):text.index("} gmm_server_trace;")]
    names = []
    for decl in re.findall(r"^\s*(?:long long|int|double)\s+([^;]+);", body, re.M):
        names += [n.strip() for n in decl.split(",")]
    assert names == [f[0] for f in G.ServerTrace._fields_]
    assert ctypes.sizeof(G.ServerTrace) == 56
    L = G.load_library()
    assert L.gmm_server_traces(None, None, 0) == 0


def test_server_stats_struct_matches_header():
    """The ctypes mirror of gmm_server_stats lists the header's fields in
    order, with C's layout."""
    text = open(os.path.join(ROOT, "include", "gmm.h")).read()
    body = text[text.index("typedef struct gmm_server_stats {"):text.index("} gmm_server_stats;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in re.findall(r"^\s*(?:long long|int|size_t|double)\s+([^;]+);", body, re.M):
        names += [n.strip() for n in decl.split(",")]
    assert names == [f[0] for f in G.ServerStats._fields_]
    assert ctypes.sizeof(G.ServerStats) == 8 * 8 + 8 + 8 * 2 + 8
