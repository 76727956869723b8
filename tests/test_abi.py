"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

from paper_1807_02587_gb300 import build_ext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    inc = os.path.join(ROOT, "include")
    txt = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s+(hgmm_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = build_ext.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ["hgmm_build", "hgmm_register", "hgmm_tree_create", "hgmm_tree_destroy",
                 "hgmm_tree_export", "hgmm_debug_labels", "hgmm_debug_reg_moments",
                 "hgmm_register_pair_host", "hgmm_sync", "hgmm_strerror",
                 "hgmm_batch_register", "hgmm_batch_features", "hgmm_mlp_forward",
                 "hgmm_mlp_train_step", "hgmm_pose_decode", "hgmm_pose_select",
                 "hgmm_register_objective", "hgmm_flat_register", "hgmm_flat_fit", "hgmm_register_descent",
                 "hgmm_debug_posteriors", "hgmm_propose", "hgmm_batch_debug_tree", "hgmm_batch_debug_root",
                 "hgmm_fit_level0_noalloc", "hgmm_batch_set_build_shape", "hgmm_batch_get_build_shape",
                 "hgmm_batch_pair_ns"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_checks(lib):
    from paper_1807_02587_gb300 import binding as B
    assert B.hgmm_node_count(1) == 8
    assert B.hgmm_node_count(3) == 584
    assert B.hgmm_node_count(4) == 4680
    assert B.hgmm_node_count(5) == 37448
    assert B.hgmm_node_count(0) == 0
    p = B.params()
    assert (p.em_iters, p.n_min, p.precision) == (8, 8.0, 0)
    assert abs(p.lam_c - 0.01) < 1e-7
    h = ctypes.c_void_p()
    # rejected before any CUDA call
    assert B._lib.hgmm_tree_create(4, 3, ctypes.byref(h)) == B.HGMM_EINVAL
    assert B._lib.hgmm_tree_create(1000, 0, ctypes.byref(h)) == B.HGMM_EINVAL
    assert B._lib.hgmm_tree_create(1000, 6, ctypes.byref(h)) == B.HGMM_EINVAL
    assert B._lib.hgmm_build(None, None, 100, 3, 8, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_register(None, None, 100, None, 3, -1.0, None, None, None) == B.HGMM_EINVAL
    for code in range(0, -8, -1):
        assert B.strerror(code) != "unknown error"
    # proposal entry points: rejected before any CUDA call
    assert B._lib.hgmm_mlp_create(0, ctypes.byref(h)) == B.HGMM_EINVAL
    assert B._lib.hgmm_mlp_create(1 << 20, ctypes.byref(h)) == B.HGMM_EINVAL
    assert B._lib.hgmm_mlp_forward(None, None, 4, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_mlp_gradients(None, None, None, None, 4, 4, 1.0, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_pose_decode(None, None, 4, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_pose_encode(None, None, 4, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_pose_select(0, None, None, None, None, None, None, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_pose_compose(1, None, None, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_tree_features(None, None, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_batch_features(None, None, None, None, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_register_objective(None, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_debug_posteriors(None, 0, None, 0) == B.HGMM_EINVAL
    assert B._lib.hgmm_propose(None, None, None, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_batch_debug_tree(None, 0, 0, None, 0) == B.HGMM_EINVAL
    assert B._lib.hgmm_batch_debug_root(None, 0, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_batch_set_build_shape(None, 0, 4, 8, 64) == B.HGMM_EINVAL
    assert B._lib.hgmm_batch_get_build_shape(None, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_batch_pair_ns(None, None, 0) == B.HGMM_EINVAL
    assert B.HGMM_MLP_PARAMS == 256 * 1280 + 256 + 256 * 256 + 256 + 9 * 256 + 9
    d = B.hgmm_descent(B.HGMM_DESCENT_MULTIPATH, 0.01, -1.0, 0)
    assert B._lib.hgmm_register_descent(None, None, 100, None, 3, ctypes.byref(d), None, None, None) == B.HGMM_EINVAL
    # flat GMM J=n variant: rejected before any CUDA call
    assert B._lib.hgmm_flat_create(0, 16, ctypes.byref(h)) == B.HGMM_EINVAL
    assert B._lib.hgmm_flat_create(1000, 0, ctypes.byref(h)) == B.HGMM_EINVAL
    assert B._lib.hgmm_flat_from_tree(None, None, -1, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_flat_fit(None, None, 100, 1, 8.0, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_flat_register(None, None, 100, None, 3, None, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_flat_objective(None, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_flat_export(None, None, 0, None, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_flat_debug_moments(None, None, 0, None) == B.HGMM_EINVAL
    assert B._lib.hgmm_flat_sync(None, None) == B.HGMM_EINVAL


def test_build_is_sm103a_only():
    assert build_ext.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
