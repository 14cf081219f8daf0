"""The C-ABI library loads and exports every symbol include/maxss.h declares (no GPU needed:
no compute call is made), and the ABI structs have the documented sizes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "maxss.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:MSS_API\s+)?(?:mss_status|void|int64_t|int32_t|const char\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_1403_2136_gb300 as mss
    from paper_1403_2136_gb300 import build
    build.build()
    return mss.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("mss_load_genome", "mss_map_reads", "nw_align", "mss_free", "mss_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import paper_1403_2136_gb300 as mss
    names = declared_functions()
    assert sorted(mss.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_struct_sizes(lib):
    import paper_1403_2136_gb300 as mss
    assert ctypes.sizeof(mss.GenomeParams) == 16
    assert ctypes.sizeof(mss.ScoreParams) == 8
    assert ctypes.sizeof(mss.NwParams) == 24
    assert mss.HIT_DTYPE.itemsize == 32
    assert mss.ALN_DTYPE.itemsize == 24


def test_max_read_len_is_the_papers_bound():
    """"Shared memory": a (m+16)*4*5-byte profile in 49152 bytes caps m at 2432."""
    import paper_1403_2136_gb300 as mss
    text = open(HEADER).read()
    m = re.search(r"#define MSS_MAX_READ_LEN (\d+)", text)
    assert int(m.group(1)) == mss.MSS_MAX_READ_LEN == ((49152 // 20 - 16) // 16) * 16


def test_null_context_is_rejected_without_a_gpu(lib):
    # argument checks happen before any CUDA call
    assert lib.mss_get_info(None, None) == -1
    assert lib.mss_last_error()


def test_null_proposal_model_is_rejected_without_a_gpu(lib):
    import paper_1403_2136_gb300 as mss
    # argument checks of the proposal entry points happen before any CUDA call
    assert lib.mss_prop_set_pooling(None, 1) == mss.MSS_EINVAL
    assert lib.mss_prop_get_pooling(None) == -1
    assert lib.mss_prop_launch_count(None) == -1
    assert lib.mss_prop_save(None, b"/nonexistent") == mss.MSS_EINVAL
