"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects bad arguments before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2511_22793_gb300 import gsparc as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "gsparc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gsparc_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(G.LIB_PATH):
        from paper_2511_22793_gb300 import build
        build.build()
    return G.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert sorted(G.EXPORTS) == names


def _declarations():
    """name -> (return type, [parameter declarations]) of every function in include/gsparc.h."""
    txt = open(os.path.join(ROOT, "include", "gsparc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"(uint32_t|int32_t|int|const char\s*\*)\s*(gsparc_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", txt):
        params = [" ".join(p.split()) for p in m.group(3).split(",") if p.strip() and p.strip() != "void"]
        out[m.group(2)] = (" ".join(m.group(1).split()), params)
    return out


def test_binding_signatures_match_the_header(L):
    """Every binding's ctypes argument list against the header: the same number of arguments,
    the same scalar type at every scalar position, a pointer at every pointer position (a
    pointer to the named struct where the header names one), and the return type."""
    scalars = {"int32_t": ctypes.c_int32, "uint32_t": ctypes.c_uint32, "int": ctypes.c_int, "int64_t": ctypes.c_int64,
               "float": ctypes.c_float, "size_t": ctypes.c_size_t}
    structs = {"gsparc_view": G.View, "gsparc_band": G.Band, "gsparc_mlp": G.MLP,
               "gsparc_mlp_grad": G.MLPGrad, "gsparc_densify_params": G.DensifyParams,
               "size_t": ctypes.c_size_t, "float": ctypes.c_float, "int64_t": ctypes.c_int64}
    decls = _declarations()
    assert sorted(decls) == sorted(G.EXPORTS)
    for name, (ret, params) in decls.items():
        fn = getattr(L, name)
        assert len(fn.argtypes) == len(params), name
        want_ret = {"int": ctypes.c_int, "int32_t": ctypes.c_int32, "uint32_t": ctypes.c_uint32,
                    "const char *": ctypes.c_char_p,
                    "const char*": ctypes.c_char_p}[ret]
        assert fn.restype is want_ret, name
        for k, (decl, got) in enumerate(zip(params, fn.argtypes)):
            if "*" not in decl:
                ctype = decl.rsplit(" ", 1)[0].replace("const ", "")
                assert got is scalars[ctype], (name, k, decl, got)
                continue
            base = decl.split("*")[0].replace("const ", "").strip()
            if got is ctypes.c_void_p:
                assert base not in ("gsparc_view", "gsparc_band", "gsparc_mlp", "gsparc_mlp_grad",
                                    "gsparc_densify_params"), (name, k, decl)
            else:
                assert getattr(got, "_type_", None) is structs[base], (name, k, decl, got)


def test_strerror_and_tiles(L):
    assert G.strerror(G.GSPARC_ERR_TIMEOUT) == "bounded device wait expired"
    assert G.gsparc_num_tiles(G.make_view(90, 360)) == 23 * 6
    assert G.gsparc_num_tiles(G.make_view(180, 720)) == 45 * 12
    assert G.gsparc_num_tiles(G.make_view(45, 180)) == 12 * 3


def test_workspace_query_grows_with_capacity(L):
    v = G.make_view(90, 360)
    a = G.gsparc_bin_sort_workspace(v, 1000, 10_000)
    b = G.gsparc_bin_sort_workspace(v, 1000, 100_000)
    assert 0 < a < b
    # the bucket keys and their second sort buffer: 16 B per pair
    assert b - a >= 16 * 90_000 - 512   # each buffer rounded up to 256 B


def test_invalid_arguments_rejected_on_host(L):
    v = G.make_view(90, 360)
    vp = ctypes.c_void_p
    assert L.gsparc_project(ctypes.byref(v), -1, None, None, None, None, None, None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_project(ctypes.byref(v), 5, None, None, None, None, None, None) == G.GSPARC_ERR_INVALID
    bad = G.make_view(0, 360)
    assert L.gsparc_project(ctypes.byref(bad), 0, None, None, None, None, None, None) == G.GSPARC_ERR_INVALID
    out = ctypes.c_size_t(0)
    assert L.gsparc_bin_sort_workspace(ctypes.byref(v), 10, 1 << 31, ctypes.byref(out)) == \
        G.GSPARC_ERR_INVALID
    band = G.make_band(0)
    assert L.gsparc_render_fwd(ctypes.byref(v), ctypes.byref(band), 1, 0, None, vp(256), vp(256), None,
                               vp(256), None, None, None, None, None) == G.GSPARC_ERR_INVALID
    m = G.MLP()
    m.hidden = 12
    rx = (ctypes.c_float * 3)(0, 0, 0)
    assert L.gsparc_attr_mlp(10, 1, vp(256), rx, vp(256), vp(256), vp(256), ctypes.byref(m), 0,
                             vp(256), None, None) == G.GSPARC_ERR_INVALID
    m.hidden = 32
    for w in ("W1", "b1", "W2", "b2", "W3", "b3"):
        setattr(m, w, vp(256))
    # stored activations: FP32 only, 16-byte aligned
    assert L.gsparc_attr_mlp(10, 1, vp(256), rx, vp(256), vp(256), vp(256), ctypes.byref(m), G.GSPARC_BF16X2,
                             vp(256), vp(256), None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_attr_mlp(10, 1, vp(256), rx, vp(256), vp(256), vp(256), ctypes.byref(m), G.GSPARC_FP32,
                             vp(256), vp(260), None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_adam(10, vp(256), vp(256), vp(256), vp(256), ctypes.c_float(1e-3),
                         ctypes.c_float(0.9), ctypes.c_float(0.999), ctypes.c_float(1e-15), 0, None) == \
        G.GSPARC_ERR_INVALID


def test_emission_stride_and_arguments(L):
    """Per-Gaussian emission buffer: 6h + 2 floats rounded up to a multiple of 4; widths outside
    1..64 and misaligned buffers are rejected on the host."""
    assert [L.gsparc_emission_stride(h) for h in (1, 5, 8, 16, 64)] == [8, 32, 52, 100, 388]
    assert L.gsparc_emission_stride(0) == 0 and L.gsparc_emission_stride(65) == 0
    vp = ctypes.c_void_p
    rx = (ctypes.c_float * 3)(0, 0, 0)
    assert L.gsparc_emission_fwd(10, 1, 0, vp(256), rx, vp(256), vp(256), vp(256), 1, vp(256), None) == \
        G.GSPARC_ERR_INVALID
    assert L.gsparc_emission_fwd(10, 1, 16, vp(256), rx, vp(256), vp(256), vp(264), 1, vp(256), None) == \
        G.GSPARC_ERR_INVALID
    assert L.gsparc_emission_bwd(10, 1, 16, vp(256), rx, vp(256), vp(256), vp(256), 1, None, vp(256), vp(256),
                                 vp(256), None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_emission_fwd(70_000_000, 1, 16, vp(256), rx, vp(256), vp(256), vp(256), 1, vp(256),
                                 None) == G.GSPARC_ERR_INVALID


def test_spectrum_loss_workspace_and_arguments(L):
    """Magnitude-spectrum loss: workspace 44 B per pixel and plane (rounded) + 256; lambda outside
    [0, 1], missing buffers and a too-small workspace are rejected on the host."""
    out = ctypes.c_size_t(0)
    assert L.gsparc_spectrum_loss_workspace(1, 64, 90, 360, ctypes.byref(out)) == 0
    n = 64 * 90 * 360
    assert out.value >= 44 * n + 256 and out.value < 44 * n + 256 + 1024
    assert L.gsparc_spectrum_loss_workspace(0, 64, 90, 360, ctypes.byref(out)) == G.GSPARC_ERR_INVALID
    vp = ctypes.c_void_p
    f32 = ctypes.c_float
    assert L.gsparc_spectrum_loss(1, 1, 8, 8, vp(256), vp(256), f32(1.5), vp(256), 1 << 20, vp(256), None,
                                  None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_spectrum_loss(1, 1, 8, 8, None, vp(256), f32(0.2), vp(256), 1 << 20, vp(256), None,
                                  None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_spectrum_loss(1, 1, 8, 8, vp(256), vp(256), f32(0.2), vp(256), 16, vp(256), None,
                                  None) == G.GSPARC_ERR_INVALID


def test_scheduled_backward_workspace_and_arguments(L):
    """Scheduled backward: workspace = 16 B header + per-(transmitter, tile) walks (rounded to
    16 B) + two 16 B items per (transmitter, tile, 64-subcarrier strip); missing or misaligned
    buffers and a too-small workspace are rejected on the host."""
    v = G.make_view(90, 360)
    T = 23 * 6
    for B, K in [(1, 64), (3, 64), (2, 128), (1, 200)]:
        strips = 1 if K <= 64 else (K + 63) // 64
        walks = (B * T * 4 + 15) // 16 * 16
        assert G.gsparc_render_bwd_tc_workspace(v, G.make_band(K), B) == 16 + walks + 2 * B * T * strips * 16
    out = ctypes.c_size_t(0)
    band = G.make_band(64)
    assert L.gsparc_render_bwd_tc_workspace(ctypes.byref(v), ctypes.byref(band), 0, ctypes.byref(out)) == \
        G.GSPARC_ERR_INVALID
    bad_band = G.make_band(0)
    assert L.gsparc_render_bwd_tc_workspace(ctypes.byref(v), ctypes.byref(bad_band), 1, ctypes.byref(out)) == \
        G.GSPARC_ERR_INVALID
    need = G.gsparc_render_bwd_tc_workspace(v, band, 1)
    vp = ctypes.c_void_p

    def call(ws=vp(4096), ws_bytes=need, d_attr=vp(4096), d_spectrum=vp(4096)):
        return L.gsparc_render_bwd_tc_balanced(ctypes.byref(v), ctypes.byref(band), 1, 10, vp(4096), vp(4096),
                                               vp(4096), vp(4096), vp(4096), None, None, vp(4096), vp(4096),
                                               d_spectrum, 0, ws, ws_bytes, d_attr, vp(4096), None, None)

    assert call(ws=None) == G.GSPARC_ERR_INVALID
    assert call(ws_bytes=need - 16) == G.GSPARC_ERR_INVALID
    assert call(d_attr=vp(4104)) == G.GSPARC_ERR_INVALID
    assert call(ws=vp(4104)) == G.GSPARC_ERR_INVALID
    assert call(d_spectrum=vp(4100)) == G.GSPARC_ERR_INVALID
    assert call(d_spectrum=None) == G.GSPARC_ERR_INVALID


def test_csi_and_fused_loss_arguments(L):
    """CSI head, channel loss and head backward reject bad sizes and misaligned complex buffers;
    the fused forward + L2 rejects a missing target, loss or gradient buffer."""
    vp = ctypes.c_void_p
    f32 = ctypes.c_float
    assert L.gsparc_csi_head(0, 4, 100, vp(256), f32(0.01), vp(256), None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_csi_head(256, 256, 100, vp(256), f32(0.01), vp(256), None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_csi_head(1, 4, 100, None, f32(0.01), vp(256), None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_csi_head(1, 4, 100, vp(260), f32(0.01), vp(256), None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_csi_loss(1, 4, vp(256), None, vp(256), None, None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_csi_loss(1, 4, vp(256), vp(256), vp(256), vp(252), None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_csi_head_bwd(1, 4, 100, vp(256), f32(0.01), None, None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_csi_head_bwd(1, 4, -1, vp(256), f32(0.01), vp(256), None) == G.GSPARC_ERR_INVALID
    v = G.make_view(90, 360)
    band = G.make_band(64)
    for target, loss, grad in [(None, vp(256), vp(256)), (vp(256), None, vp(256)), (vp(256), vp(256), None),
                               (vp(260), vp(256), vp(256))]:
        assert L.gsparc_render_fwd_l2_tc(ctypes.byref(v), ctypes.byref(band), 1, 10, vp(256), vp(256), vp(256),
                                         vp(256), target, loss, grad, vp(256), vp(256), vp(256), None, None,
                                         None, None, None) == G.GSPARC_ERR_INVALID


def test_confidence_arguments(L):
    """Confidence objective: widths outside 1..32, a negative batch, missing weights, objective,
    positions or losses, and a negative or NaN alpha are rejected on the host."""
    vp = ctypes.c_void_p
    f32 = ctypes.c_float
    ok = dict(B=4, hidden=32, pos=vp(256), loss=vp(256), w=vp(256), alpha=f32(0.3), obj=vp(256))

    def call(**kw):
        a = dict(ok, **kw)
        return L.gsparc_confidence(a["B"], a["hidden"], a["pos"], a["loss"], a["w"], a["alpha"], None,
                                   a["obj"], None, None, None)

    for bad in (dict(hidden=0), dict(hidden=33), dict(B=-1), dict(w=None), dict(obj=None), dict(pos=None),
                dict(loss=None), dict(alpha=f32(-0.1)), dict(alpha=f32(float("nan")))):
        assert call(**bad) == G.GSPARC_ERR_INVALID, bad


def test_densify_workspace_and_arguments(L):
    """Densification: 4 B of workspace per 256 Gaussians (rounded to 256 B); n_split outside 1..8,
    negative or NaN thresholds, missing inputs or outputs and a small workspace are rejected on the
    host; the opacity reset wants 0 < max_opacity < 1."""
    assert G.gsparc_densify_workspace(0) == 0
    assert G.gsparc_densify_workspace(1) == 256
    assert G.gsparc_densify_workspace(256 * 64) == 256
    assert G.gsparc_densify_workspace(256 * 65) == 512
    vp = ctypes.c_void_p
    good = G.densify_params()
    need = G.gsparc_densify_workspace(1000)

    def call(params=good, N=1000, P=4, cap=3000, ws=vp(4096), ws_bytes=need, payload=vp(4096), out_means=vp(4096),
             xi=vp(4096), n_out=vp(4096)):
        return L.gsparc_densify(N, P, vp(4096), vp(4096), vp(4096), vp(4096), payload, vp(4096), vp(4096), vp(4096),
                                xi, ctypes.byref(params), cap, ws, ws_bytes, out_means, vp(4096), vp(4096), vp(4096),
                                vp(4096), vp(4096), n_out, None, None)

    for field, value in (("n_split", 0), ("n_split", 9), ("tau_grad", -1.0), ("r_max", float("nan")),
                         ("sigma_min", -0.1), ("clone_scale", float("nan"))):
        bad = G.densify_params()
        setattr(bad, field, value)
        assert call(params=bad) == G.GSPARC_ERR_INVALID, field
    assert call(N=-1) == G.GSPARC_ERR_INVALID
    assert call(cap=-1) == G.GSPARC_ERR_INVALID
    assert call(payload=None) == G.GSPARC_ERR_INVALID
    assert call(xi=None) == G.GSPARC_ERR_INVALID
    assert call(out_means=None) == G.GSPARC_ERR_INVALID
    assert call(n_out=None) == G.GSPARC_ERR_INVALID
    assert call(ws_bytes=need - 1) == G.GSPARC_ERR_WORKSPACE
    assert call(ws=None) == G.GSPARC_ERR_WORKSPACE
    assert call(ws=vp(4098)) == G.GSPARC_ERR_INVALID
    f32 = ctypes.c_float
    for m in (0.0, 1.0, -0.5, float("nan")):
        assert L.gsparc_opacity_reset(10, f32(m), vp(4096), None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_opacity_reset(10, f32(0.01), None, None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_densify_accumulate(10, vp(4096), None, vp(4096), vp(4096), None) == G.GSPARC_ERR_INVALID
    assert L.gsparc_densify_accumulate(-1, vp(4096), vp(4096), vp(4096), vp(4096), None) == G.GSPARC_ERR_INVALID


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(G, "_lib", None)
    monkeypatch.setattr(G, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        G.lib()


def test_wrappers_pass_arguments_in_header_order(monkeypatch):
    """The Python wrappers of the training extras, the spectrum loss and the emission network
    marshal every tensor to the header parameter of the same meaning, in order, and derive the
    sizes from the tensors' shapes (host only: the C call is recorded, not made)."""
    import torch

    decls = _declarations()
    calls = []
    names = {}

    def t(name, *shape, dtype=torch.float32):
        x = torch.zeros(shape, dtype=dtype)
        names[id(x)] = name
        return x

    monkeypatch.setattr(G, "_p", lambda x: None if x is None else names[id(x)])
    monkeypatch.setattr(G, "_stream", lambda s=None: "stream")
    monkeypatch.setattr(G, "_call", lambda fn, *args: calls.append((fn, args)))

    def check(expect_sizes):
        fn, args = calls.pop()
        params = [p.split()[-1].lstrip("*") for p in decls[fn][1]]
        assert len(args) == len(params), fn
        for p, a in zip(params, args):
            if p in expect_sizes:
                assert a == expect_sizes[p], (fn, p, a)
            elif isinstance(a, str):
                assert a == p, (fn, p, a)

    G.gsparc_confidence(t("pos", 5, 3), t("task_loss", 5), t("weights", 161), 32, t("objective", 1),
                        t("confidence", 5), t("d_task_loss", 5), t("d_weights", 161), alpha=0.25)
    check({"B": 5, "hidden": 32, "alpha": 0.25})
    out = {"means": t("out_means", 9, 3), "log_scales": t("out_log_scales", 9, 3), "quats": t("out_quats", 9, 4),
           "opacity_logit": t("out_opacity_logit", 9), "payload": t("out_payload", 9, 2),
           "parent": t("out_parent", 9, dtype=torch.int32)}
    params = G.densify_params()
    G.gsparc_densify(t("means", 4, 3), t("log_scales", 4, 3), t("quats", 4, 4), t("opacity_logit", 4),
                     t("payload", 4, 2), t("proj", 4, 8), t("norm_sum", 4), t("count", 4, dtype=torch.int32),
                     t("xi", 4, 2, 3), params, t("ws", 256, dtype=torch.uint8), out,
                     t("n_out", 1, dtype=torch.int32), t("d_status", 1, dtype=torch.int32))
    fn, args = calls[-1]
    assert args[11]._obj is params
    check({"N": 4, "P": 2, "capacity": 9, "ws_bytes": 256, "params": args[11]})
    G.gsparc_densify_accumulate(t("proj", 6, 8), t("d_means", 6, 3), t("norm_sum", 6), t("count", 6))
    check({"N": 6})
    G.gsparc_opacity_reset(t("opacity_logit", 7), 0.02)
    check({"N": 7, "max_opacity": 0.02})
    G.gsparc_spectrum_loss(t("spectrum", 2, 3, 4, 5, 2), t("target", 2, 3, 4, 5), t("ws", 512, dtype=torch.uint8),
                           t("loss", 1), t("d_spectrum", 2, 3, 4, 5, 2), lam=0.3)
    check({"B": 2, "K": 3, "H": 4, "W": 5, "lambda": 0.3, "ws_bytes": 512})
    G.gsparc_emission_fwd(t("tx", 3, 3), (0.0, 1.0, 2.0), t("means", 8, 3), t("opacity_logit", 8),
                          t("weights", 8, 100), 16, t("attr", 3, 8, 4), inv_d=False)
    fn, args = calls[-1]
    assert list(args[4]) == [0.0, 1.0, 2.0]
    check({"N": 8, "B": 3, "hidden": 16, "rx": args[4], "inv_d": 0})
    G.gsparc_emission_bwd(t("tx", 2, 3), (0.5, 0.0, 0.0), t("means", 8, 3), t("opacity_logit", 8),
                          t("weights", 8, 100), 16, t("d_attr", 2, 8, 4), t("d_means", 8, 3),
                          t("d_opacity_logit", 8), t("d_weights", 8, 100))
    fn, args = calls[-1]
    check({"N": 8, "B": 2, "hidden": 16, "rx": args[4], "inv_d": 1})


def test_overlap_groups_match_the_header():
    txt = open(os.path.join(ROOT, "include", "gsparc.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (GSPARC_OVERLAP_[A-Z_]+) (\d+)", txt)}
    assert len(defs) == 6
    for name, v in defs.items():
        assert getattr(G, name) == v, name
    groups = [v for n, v in defs.items() if n != "GSPARC_OVERLAP_ALL"]
    assert sum(groups) == defs["GSPARC_OVERLAP_ALL"] and all(g & (g - 1) == 0 for g in groups)
