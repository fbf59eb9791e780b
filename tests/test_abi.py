"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/s3r.h declares (no compute calls here)."""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "s3r.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(s3r_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("s3r_project", "s3r_sort", "s3r_render_fwd", "s3r_render_bwd",
                     "s3r_update_visibility"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2503_08217_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.s3r_built_arch.restype = ctypes.c_int32
    assert lib.s3r_built_arch() == 103


def test_binding_lists_every_declared_symbol():
    from paper_2503_08217_gb300 import binding
    assert set(binding.EXPORTS) == set(declared_functions())


def test_invalid_calls_fail_without_a_gpu():
    """Argument checks run before any CUDA call: NULL handles are rejected."""
    from paper_2503_08217_gb300 import binding
    L = binding.load()
    assert L.s3r_sort(None, None) == 1
    assert L.s3r_render_fwd(None, None, None, None) == 1
    assert L.s3r_update_visibility(-1, 0.0, None, None, None, 0, None) == 1
    assert L.s3r_update_visibility(10, 0.0, None, None, None, 7, None) == 1
    assert b"mode" in L.s3r_last_error()
    assert L.s3r_check_wait_timeout(None, 100, None) == 1
    assert L.s3r_set_epoch(None, 5, None) == 1
    assert b"workspace" in L.s3r_last_error()
    assert L.s3r_device_status(None) is None


def test_adam_argument_checks_fail_without_a_gpu():
    """s3r_adam_step validates its descriptors before any launch."""
    from paper_2503_08217_gb300 import binding
    L = binding.load()
    T = binding.AdamTensor
    arr = (T * 9)()
    assert L.s3r_adam_step(arr, 9, 1e-3, 0.9, 0.999, 1e-8, 1, None, None) == 1     # > 8 tensors
    assert L.s3r_adam_step(arr, 1, 1e-3, 0.9, 0.999, 1e-8, 0, None, None) == 1     # step 0
    assert L.s3r_adam_step(arr, 1, 1e-3, 1.0, 0.999, 1e-8, 1, None, None) == 1     # beta1 = 1
    arr[0] = T(None, None, None, None, 10)
    assert L.s3r_adam_step(arr, 1, 1e-3, 0.9, 0.999, 1e-8, 1, None, None) == 1     # NULL arrays
    assert b"adam" in L.s3r_last_error()


def test_set_lod_rejects_a_null_workspace_without_a_gpu():
    from paper_2503_08217_gb300 import binding
    L = binding.load()
    prm = binding.LodParams(binding.LOD_STOCHASTIC, 0.5, 10.0, (0.1, 0.1, 0.1), 7)
    assert L.s3r_set_lod(None, prm) == 1


def test_to_world_rejects_bad_arguments_without_a_gpu():
    """s3r_to_world validates the scene, poses and outputs before any CUDA call."""
    from paper_2503_08217_gb300 import binding
    L = binding.load()
    sc = binding.Scene()
    sc.n = 10
    sc.n_inst = 1
    poses = binding.Poses()
    assert L.s3r_to_world(None, ctypes.byref(poses), None, None, None, None) == 1     # NULL scene
    assert L.s3r_to_world(ctypes.byref(sc), ctypes.byref(poses), None, None, None, None) == 1   # no offsets
    assert b"inst_offsets" in L.s3r_last_error()
    offs = (ctypes.c_int64 * 3)(0, 5, 10)
    sc.inst_offsets = ctypes.cast(offs, ctypes.c_void_p)
    assert L.s3r_to_world(ctypes.byref(sc), ctypes.byref(poses), None, None, None, None) == 1   # no arrays
    assert b"required" in L.s3r_last_error()


def test_to_world_bwd_rejects_a_null_workspace_without_a_gpu():
    from paper_2503_08217_gb300 import binding
    L = binding.load()
    assert L.s3r_to_world_bwd(None, None, None, None, None) == 1
    assert b"workspace" in L.s3r_last_error()
