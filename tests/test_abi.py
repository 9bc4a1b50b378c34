"""The C-ABI library loads and exports every entry point its header declares
(host-only checks, no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "leysort.h")


@pytest.fixture(scope="module")
def ley():
    from paper_1909_08006_gb300 import build
    build.build()
    import paper_1909_08006_gb300 as m
    return m


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ley_[a-z_]+)\s*\(", text)))


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header alone compiles as C99, with no C++
    # or PyTorch types
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text('#include "leysort.h"\nint main(void) { return 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-fsyntax-only", "-I", os.path.dirname(HEADER), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ley_sort_records", "ley_sort_keys_index", "ley_partition_records",
                     "ley_workspace_bytes", "ley_status_string", "ley_last_device_status"]:
        assert required in names


def test_library_exports_every_declared_symbol(ley):
    lib = ctypes.CDLL(ley.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in leysort.h but not exported"
    for name in ley.exported_symbols():
        assert name in declared_functions(), f"binding names {name}, header does not"


def test_host_only_entry_points(ley):
    assert ley.ley_status_string(ley.LEY_OK) == "ok"
    assert "budget" in ley.ley_status_string(ley.LEY_ENOMEM)
    assert ley.ley_status_string(99) == "unknown status"
    assert ley.ley_workspace_bytes(0) == 0
    b = ley.ley_workspace_bytes(100_000_000)
    # 100-byte records are gathered inside the finishing kernel: two 16-byte
    # tuple buffers per record, plus control
    assert 32 * 100_000_000 < b < 38 * 100_000_000
    # other record sizes also hold a 4-byte permutation per record
    b104 = ley.ley_workspace_bytes(100_000_000, rec_bytes=104)
    assert b104 - b == 4 * 100_000_000
    with pytest.raises(ley.LeyError) as e:
        ley.ley_workspace_bytes(10, rec_bytes=100, key_bytes=101)
    assert e.value.status == ley.LEY_EUNSUPPORTED
    # keys longer than 12 bytes: a permutation and two order arrays more
    assert ley.ley_workspace_bytes(100_000_000, key_bytes=30) > b + 12 * 100_000_000 - 1
    # any record size from key_bytes to 4096 bytes (not only multiples of 4)
    assert ley.ley_workspace_bytes(100_000_000, rec_bytes=102) == b104
    assert ley.ley_workspace_bytes(1000, rec_bytes=10, key_bytes=10) > 0
    assert ley.ley_workspace_bytes(1000, rec_bytes=1, key_bytes=1) > 0
    with pytest.raises(ley.LeyError) as e:
        ley.ley_workspace_bytes(10, rec_bytes=4097, key_bytes=10)
    assert e.value.status == ley.LEY_EUNSUPPORTED


def test_workspace_bytes_under_a_budget(ley):
    # host-memory sorts under a device budget (Section 4.1's 20 GB partially
    # in-memory and 60 GB external data sets under a 30 GB limit)
    budget = 30_000_000_000
    n = 200_000_000
    part = ley.ley_workspace_bytes(n, mem_budget=budget)
    internal = ley.ley_workspace_bytes(n, rec_bytes=104)  # with the permutation
    # the partial mode holds the input, one workspace and four staging buffers
    assert n * 100 + internal <= part <= n * 100 + internal + 4 * (64 << 20) + 4096
    assert part <= budget
    n = 600_000_000
    ext = ley.ley_workspace_bytes(n, mem_budget=budget)
    assert 0 < ext <= budget  # the external mode's rotating buffers fit the cap
    assert ext < n * 100
    # a budget that holds no mode at all
    with pytest.raises(ley.LeyError) as e:
        ley.ley_workspace_bytes(n, mem_budget=1 << 20)
    assert e.value.status == ley.LEY_ENOMEM
    # the budget never changes the answer for the internal sort of device
    # buffers (mem_budget 0), and n == 0 needs nothing
    assert ley.ley_workspace_bytes(0, mem_budget=budget) == 0
    # pinned host scratch: none in the partial mode; in the external mode the
    # runs that do not stay on the device (a 30 GB budget keeps several of
    # the 18.75M-record runs of 6e8 records there)
    assert ley.ley_host_scratch_bytes(200_000_000, mem_budget=budget) == 0
    hb = ley.ley_host_scratch_bytes(600_000_000, mem_budget=budget)
    assert 0 < hb < 600_000_000 * 100 and hb % (100 * 4096) == 0
    # a smaller budget keeps fewer runs on the device, never more than it holds
    hb10 = ley.ley_host_scratch_bytes(600_000_000, mem_budget=10_000_000_000)
    assert hb < hb10 < 600_000_000 * 100 and hb10 >= 600_000_000 * 100 - 10_000_000_000
    assert hb >= 600_000_000 * 100 - budget
    # with no runs kept on the device every run goes to the host
    import os
    os.environ["LEY_EXTERNAL_RESIDENT"] = "0"
    try:
        assert ley.ley_host_scratch_bytes(600_000_000, mem_budget=budget) == 600_000_000 * 100
    finally:
        del os.environ["LEY_EXTERNAL_RESIDENT"]
    with pytest.raises(ley.LeyError) as e:
        ley.ley_host_scratch_bytes(600_000_000, mem_budget=1 << 20)
    assert e.value.status == ley.LEY_ENOMEM


def test_argument_checks_before_any_gpu_work(ley):
    # geometry and size checks happen before memory kinds are inspected
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records(0, 0, n=10, rec_bytes=100, key_bytes=0)
    assert e.value.status == ley.LEY_EUNSUPPORTED
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records(0, 0, n=1 << 32, rec_bytes=100, key_bytes=10)
    assert e.value.status == ley.LEY_EUNSUPPORTED
    # n == 0 is a no-op that touches nothing
    assert ley.ley_sort_records(0, 0, n=0, rec_bytes=100, key_bytes=10) == ley.LEY_OK
    assert ley.ley_sort_keys_index(0, 0, 0, 0, n=0) == ley.LEY_OK
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records(0, 0, n=5, rec_bytes=100, key_bytes=10)
    assert e.value.status == ley.LEY_EINVAL
    # the queued variant checks its arguments the same way
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records_async(0, 0, n=10, rec_bytes=100, key_bytes=0)
    assert e.value.status == ley.LEY_EUNSUPPORTED
    assert ley.ley_sort_records_async(0, 0, n=0, rec_bytes=100, key_bytes=10) == ley.LEY_OK
    with pytest.raises(ley.LeyError) as e:
        ley.ley_sort_records_async(0, 0, n=5, rec_bytes=100, key_bytes=10)
    assert e.value.status == ley.LEY_EINVAL


def test_launch_counter_and_profiler_are_host_state(ley):
    assert ley.ley_launch_count() >= 0
    ley.ley_profile_enable(True)
    assert ley.ley_profile_read() == {}
    ley.ley_profile_enable(False)
