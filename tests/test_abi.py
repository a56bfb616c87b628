"""C-ABI checks that need no GPU: the library loads, exports every entry
point that include/*.h declares, rejects bad descriptors on the host, and
shares no code with the oracle."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1309_0052_b300 import build as b
    b.build()
    import paper_1309_0052_b300 as g
    return g


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"^GNSS_API\s+[\w\s\*]+?\b(gnss_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("gnss_plan_create", "gnss_plan_destroy", "gnss_acquire", "gnss_acquire_device",
                 "gnss_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib.lib, name), name


def test_internal_symbols_are_hidden(lib):
    # only the C ABI is exported (the library is built with -fvisibility=hidden)
    with pytest.raises(AttributeError):
        getattr(lib.lib, "_ZN4gnss9set_errorERKNSt7__cxx1112basic_stringIcSt11char_traitsIcESaIcEEE")


@pytest.mark.parametrize("field,value", [("fs_hz", 4095000), ("fs_hz", 3000000), ("fs_hz", 128000),
                                         ("fs_hz", 32768000), ("coh_ms", 0), ("n_dopp", 0),
                                         ("prn_mask", 0), ("prn_mask", 1 << 32), ("format", 7),
                                         ("flags", 0x80), ("dopp_step_hz", 0)])
def test_bad_descriptor_rejected_on_host(lib, field, value):
    d = lib.PlanDesc(fs_hz=2048000, coh_ms=1, noncoh=0, dopp_min_hz=-5000, dopp_step_hz=500, n_dopp=21,
                     prn_mask=0xFFFFFFFF, threshold=2.0, flags=0, format=0)
    setattr(d, field, value)
    h = C.c_void_p()
    st = lib.lib.gnss_plan_create(C.byref(d), C.byref(h))
    assert st == lib.EINVAL
    assert not h.value
    assert lib.lib.gnss_last_error()


def test_recording_bytes(lib):
    assert lib.recording_bytes(lib.FMT_I8_IQ, 8192) == 16384
    assert lib.recording_bytes(lib.FMT_2BIT_IQ, 409600) == 204800
    assert lib.recording_bytes(lib.FMT_2BIT_IQ, 3) == 2


def test_null_arguments_rejected(lib):
    h = C.c_void_p()
    assert lib.lib.gnss_plan_create(None, C.byref(h)) == lib.EINVAL
    assert lib.lib.gnss_plan_destroy(None) == lib.OK
    assert lib.lib.gnss_acquire(None, None, 0, 0, None, None, None) == lib.EINVAL


def test_oracle_and_cuda_path_share_no_code():
    """The oracle (test infrastructure) and the product share no source: no
    include, import or file reference crosses between them."""
    pkg = os.path.join(ROOT, "paper_1309_0052_b300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            src = open(path).read()
            assert "import oracle" not in src and "from oracle" not in src and "oracle.c" not in src and "liboracle" not in src, path
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.*")):
        if path.endswith((".py", ".c", ".h")):
            src = open(path).read()
            assert "paper_1309_0052_b300" not in src and "gnss.h" not in src and "csrc" not in src, path


def test_host_side_rejections_of_later_entry_points(lib):
    L = lib.lib
    E = lib.EINVAL
    assert L.gnss_refine(None, None, 0, 0, None, 1, 10, 10, 0.0, None, None) == E
    assert L.gnss_refine_device(None, None, 0, None, 1, 10, 10, 0.0, None, None) == E
    assert L.gnss_refine_eval(None, None, 0, 10, None, None, None, 1, None, None, None, None) == E
    assert L.gnss_acquire_batch(None, 1, 0, None) == E
    assert L.gnss_acquire_batch(None, 0, 0, None) == lib.OK  # empty batch
    assert L.gnss_autotune(None, 0, None) == E
    assert L.gnss_submit(None, None, None, 0, None) == E
    assert L.gnss_poll(None, 1, None, 0, None) == E
    assert L.gnss_wait(None, 1, 0, None, 0, None) == E
    assert L.gnss_cancel(None, 1) == E
    assert L.gnss_server_get_stats(None, None) == E
    assert L.gnss_server_destroy(None) == lib.OK
    fn = L.gnss_acquire_noalloc
    fn.argtypes = [C.c_void_p] * 3 + [C.c_void_p] * 3
    assert fn(None, None, 0, None, None, None) == E
    # traced acquisition: NULL events or outputs are rejected before any device work
    assert L.gnss_acquire_device_traced(None, None, 0, None, None, None, None) == E
    # batch graph: NULL handle slot, NULL graph; destroying NULL is a no-op
    h = C.c_void_p()
    assert L.gnss_batch_graph_create(None, 1, 0, None) == E
    assert L.gnss_batch_graph_create(None, 0, 0, C.byref(h)) == E and not h.value
    assert L.gnss_batch_graph_launch(None, None) == E
    assert L.gnss_batch_graph_destroy(None) == lib.OK
    cfg = lib.TrackConfig(1, 10, 1.0, 15.0, 1.0, 0)
    assert L.gnss_track(None, None, 0, None, 1, C.byref(cfg), None, None) == E


def test_record_layouts_match_the_header(lib, tmp_path):
    """sizeof / offsetof of the header's records, compiled by gcc, equal the
    binding's ctypes / numpy layouts."""
    import subprocess
    src = tmp_path / "sizes.c"
    src.write_text(r"""
#include <stddef.h>
#include <stdio.h>
#include "gnss.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(gnss_plan_desc), sizeof(gnss_detection),
         sizeof(gnss_candidate), sizeof(gnss_refined), sizeof(gnss_request), sizeof(gnss_server_config),
         sizeof(gnss_server_stats), sizeof(gnss_tune_result), sizeof(gnss_plan_info), sizeof(gnss_track_config),
         sizeof(gnss_track_rec));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(gnss_detection, dopp_bin), offsetof(gnss_detection, ratio),
         offsetof(gnss_refined, status), offsetof(gnss_plan_desc, prn_mask), offsetof(gnss_track_rec, zl),
         offsetof(gnss_track_rec, status));
  return 0;
}
""")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sizes, offs = [list(map(int, l.split())) for l in subprocess.check_output([str(exe)]).decode().splitlines()]
    assert sizes == [C.sizeof(lib.PlanDesc), lib.DETECTION_DTYPE.itemsize, lib.CANDIDATE_DTYPE.itemsize,
                     lib.REFINED_DTYPE.itemsize, C.sizeof(lib.Request), C.sizeof(lib.ServerConfig),
                     C.sizeof(lib.ServerStats), C.sizeof(lib.TuneResult), C.sizeof(lib.PlanInfo),
                     C.sizeof(lib.TrackConfig), lib.TRACK_DTYPE.itemsize]
    assert offs == [lib.DETECTION_DTYPE.fields["dopp_bin"][1], lib.DETECTION_DTYPE.fields["ratio"][1],
                    lib.REFINED_DTYPE.fields["status"][1], lib.PlanDesc.prn_mask.offset,
                    lib.TRACK_DTYPE.fields["zl"][1], lib.TRACK_DTYPE.fields["status"][1]]
