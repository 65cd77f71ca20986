"""The C-ABI library builds, loads and exports every declared symbol (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "twopaco.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(twopaco_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("twopaco_build", "twopaco_build_ex", "twopaco_result_free", "twopaco_strerror",
                 "twopaco_run_device", "twopaco_workspace_size", "twopaco_read_stats"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1602_05856_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_checks():
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    assert T.twopaco_strerror(T.EINVAL) == "invalid argument"
    ok = T.twopaco_workspace_size(1000, 2, 25, 1 << 20, 1)
    assert ok > (1 << 20) // 8
    bad = [dict(k=0), dict(k=128), dict(filter_bits=100), dict(filter_bits=3 << 10), dict(rounds=0),
           dict(options=T.Options(hashes=0)), dict(options=T.Options(hashes=9)),
           dict(options=T.Options(partition_bins=1000)), dict(rounds=8, options=T.Options(partition_bins=4)),
           dict(options=T.Options(wide_layout=3)), dict(options=T.Options(wide_layout=-1)),
           dict(options=T.Options(split_at_n=True, run_capacity=1 << 32)),
           dict(filter_bits=1 << 41), dict(n_seqs=1 << 32), dict(rounds=2, options=T.Options(partition_bins=1)),
           dict(options=T.Options(bucket_inserts=3)), dict(options=T.Options(bucket_inserts=-1))]
    for b in bad:
        args = dict(total_bases=1000, n_seqs=2, k=25, filter_bits=1 << 20, rounds=1)
        args.update(b)
        with pytest.raises(T.TwopacoError) as e:
            T.twopaco_workspace_size(**args)
        assert e.value.code == T.EINVAL
    # a null workspace is rejected before anything is launched
    with pytest.raises(T.TwopacoError) as e:
        T.twopaco_run_device(0, 0, 0, 0, 25, 1 << 20, 1, None, 0, 0, 0, 0, 0)
    assert e.value.code == T.EINVAL


def test_workspace_grows_with_input_and_filter():
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    a = T.twopaco_workspace_size(10**6, 4, 25, 1 << 20, 1)
    b = T.twopaco_workspace_size(10**7, 4, 25, 1 << 20, 1)
    c = T.twopaco_workspace_size(10**6, 4, 25, 1 << 26, 1)
    d = T.twopaco_workspace_size(10**6, 4, 63, 1 << 20, 1)
    assert b > a and c - a >= ((1 << 26) - (1 << 20)) // 8 and d > a


def test_split_and_long_k_workspace():
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    plain = T.twopaco_workspace_size(1 << 20, 4, 25, 1 << 20, 1)
    split = T.twopaco_workspace_size(1 << 20, 4, 25, 1 << 20, 1, T.Options(split_at_n=True))
    assert split > plain + 2 * ((1 << 20) // 8)  # N mask and boundary bitmap
    small = T.twopaco_workspace_size(1 << 20, 4, 25, 1 << 20, 1, T.Options(split_at_n=True, run_capacity=16))
    assert plain < small < split
    assert T.twopaco_workspace_size(1 << 20, 4, 100, 1 << 20, 1) > 0
    assert T.twopaco_workspace_size(1 << 20, 4, 127, 1 << 20, 1) > 0


def test_wide_layout_workspace():
    """64-bit records need no more room than the 32-bit ones (the list holds
    half as many), and drop the probe descriptors (8 B per base) and, at 2,
    the kept slots; from 2^31 bases the automatic layout is already wide."""
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    m = 1 << 24
    w0, w1, w2 = (T.twopaco_workspace_size(m, 10, 25, 1 << 26, 1, T.Options(wide_layout=w)) for w in (0, 1, 2))
    assert w0 - w1 >= 8 * m and w1 - w2 >= 4 * (m // 2)
    big = 1 << 31
    b0, b1 = (T.twopaco_workspace_size(big, 10, 25, 1 << 26, 1, T.Options(wide_layout=w)) for w in (0, 1))
    assert b0 == b1


def test_checkpoint_sizes_and_round_range_checks():
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    m = 1 << 20
    one = T.twopaco_checkpoint_bytes(m, 3, 25, 1 << 20, 1)
    four = T.twopaco_checkpoint_bytes(m, 3, 25, 1 << 20, 4, T.Options(partition_bins=1024))
    assert one >= m // 8 and four == one + 3 * 4 + 1024 * 4
    for b, e in ((-1, 1), (0, 0), (2, 1), (0, 5)):  # rounds = 4
        with pytest.raises(T.TwopacoError) as err:
            T.twopaco_run_rounds(0, 0, 0, 0, 25, 1 << 20, 4, T.Options(partition_bins=64), 0, 0,
                                 b, e, 0, 0, 0)
        assert err.value.code == T.EINVAL


def test_kernel_code_digest_follows_code_not_comments(tmp_path, monkeypatch):
    """The ncu traffic figures bench.py reports are keyed to the kernel code only."""
    import os
    import shutil
    import bench
    src = os.path.join(bench.ROOT, "paper_1602_05856_gb300", "csrc", "twopaco_kernels.cu")
    d = tmp_path / "paper_1602_05856_gb300" / "csrc"
    d.mkdir(parents=True)
    shutil.copy(src, d / "twopaco_kernels.cu")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.kernel_code_digest()
    text = (d / "twopaco_kernels.cu").read_text()
    (d / "twopaco_kernels.cu").write_text("// a new comment\n\n" + text.replace("{\n", "{  /* note */\n", 1))
    assert bench.kernel_code_digest() == base
    (d / "twopaco_kernels.cu").write_text(text.replace("kInsertR = 16", "kInsertR = 8", 1))
    assert bench.kernel_code_digest() != base
    assert bench.ncu_traffic("bacterial_set", "pass1_insert") is None  # no profiles under tmp_path


def test_checkpoint_checksum_detects_changes(tmp_path):
    """The payload checksum of a checkpoint (host code, built here with g++):
    any flipped bit, two swapped words or another length change it."""
    import subprocess
    src = tmp_path / "sum.cpp"
    src.write_text(r'''
#include <cstdio>
#include <vector>
#include "twopaco_checksum.h"
int main() {
  std::vector<unsigned char> b(1003);
  for (size_t i = 0; i < b.size(); ++i) b[i] = (unsigned char)(i * 131 + 7);
  const uint64_t base = twopaco::payload_checksum(b.data(), b.size());
  int bad = 0;
  for (size_t i = 0; i < b.size(); ++i)
    for (int bit = 0; bit < 8; ++bit) {
      b[i] ^= (unsigned char)(1 << bit);
      bad += twopaco::payload_checksum(b.data(), b.size()) == base;
      b[i] ^= (unsigned char)(1 << bit);
    }
  std::vector<unsigned char> s = b;
  for (int j = 0; j < 8; ++j) std::swap(s[j], s[8 + j]);
  bad += twopaco::payload_checksum(s.data(), s.size()) == base;
  bad += twopaco::payload_checksum(b.data(), b.size() - 1) == base;
  std::vector<unsigned char> z(b);
  z.push_back(0);
  bad += twopaco::payload_checksum(z.data(), z.size()) == base;
  bad += twopaco::payload_checksum(b.data(), b.size()) != base;
  std::printf("%d %llu\n", bad, (unsigned long long)twopaco::payload_checksum("", 0));
  return 0;
}
''')
    csrc = os.path.join(ROOT, "paper_1602_05856_gb300", "csrc")
    exe = tmp_path / "sum"
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", csrc, str(src), "-o", str(exe)], check=True)
    bad, _ = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert bad == "0"


def test_partial_option_checks_and_smaller_workspace():
    """partial is 0 or 1; without the second pass the workspace holds no table, list
    or kept slots."""
    import ctypes
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    o = T.Options()._c()
    o.partial = 2
    b = ctypes.c_uint64(0)
    rc = T.load().twopaco_workspace_size(1000, 2, 25, 1 << 20, 1, ctypes.byref(o), ctypes.byref(b))
    assert rc == T.EINVAL
    m = 10**7
    full = T.twopaco_workspace_size(m, 4, 25, 1 << 24, 1)
    part = T.twopaco_workspace_size(m, 4, 25, 1 << 24, 1, T.Options(partial=True))
    table = 8 * (1 << 25)  # next power of two of 2m one-word slots
    assert full - part >= table


def test_bucketed_inserts_follow_the_or_density():
    """Automatic region buckets only where a chunk puts >= 16 ORs on each filter sector."""
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    ws = lambda m, bits, b, r=1: T.twopaco_workspace_size(m, 8, 25, bits, r, T.Options(bucket_inserts=b))
    assert ws(310_000_000, 1 << 30, 0) > ws(310_000_000, 1 << 30, 2)      # 77 ORs per sector
    assert ws(24_000_000_000, 1 << 36, 0, 4) == ws(24_000_000_000, 1 << 36, 2, 4)  # about 7
    assert ws(35_000_000, 1 << 28, 0) == ws(35_000_000, 1 << 28, 2)       # within L2
    assert ws(35_000_000, 1 << 28, 1) > ws(35_000_000, 1 << 28, 2)        # forced


def test_launch_shape_option_range():
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    for bad in (-1, 33):
        with pytest.raises(T.TwopacoError) as e:
            T.twopaco_workspace_size(1000, 2, 25, 1 << 20, 1, T.Options(launch_blocks_per_sm=bad))
        assert e.value.code == T.EINVAL
    assert T.twopaco_workspace_size(1000, 2, 25, 1 << 20, 1, T.Options(launch_blocks_per_sm=2)) == \
        T.twopaco_workspace_size(1000, 2, 25, 1 << 20, 1)


def test_ordered_first_pass_layout():
    """The region-ordered first pass: automatic for class-map runs with a filter of
    1 GiB and more, forced on any class-map run, never without a class map, for
    k > 63 or more than 6 bits per item; the option takes 0, 1 or 2."""
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    for bad in (-1, 3):
        with pytest.raises(T.TwopacoError) as e:
            T.twopaco_workspace_size(1000, 2, 25, 1 << 20, 2, T.Options(ordered_first_pass=bad))
        assert e.value.code == T.EINVAL

    def ws(m, bits, rounds, o, k=25, h=4, **kw):
        return T.twopaco_workspace_size(m, 8, k, bits, rounds, T.Options(hashes=h, ordered_first_pass=o, **kw))

    big = 24_000_000_000
    # a region byte per position and 8-byte records for a round and a quarter, which
    # hold the candidate list (by default half a round of 8-byte records)
    per_round = big // 4
    assert ws(big, 1 << 36, 4, 0) - ws(big, 1 << 36, 4, 2) >= big + 8 * (per_round * 5 // 4) - 8 * (per_round // 2)
    assert ws(big, 1 << 36, 4, 0) == ws(big, 1 << 36, 4, 1)
    assert ws(35_000_000, 1 << 28, 4, 0) == ws(35_000_000, 1 << 28, 4, 2)   # 32 MiB: within L2
    assert ws(35_000_000, 1 << 28, 4, 1) > ws(35_000_000, 1 << 28, 4, 2)    # forced
    assert ws(35_000_000, 1 << 28, 1, 1) == ws(35_000_000, 1 << 28, 1, 2)   # one round: no class map
    assert ws(35_000_000, 1 << 28, 4, 1, k=100) == ws(35_000_000, 1 << 28, 4, 2, k=100)
    assert ws(35_000_000, 1 << 28, 4, 1, h=7) == ws(35_000_000, 1 << 28, 4, 2, h=7)
    assert ws(35_000_000, 1 << 28, 4, 1, per_string_launches=True) == \
        ws(35_000_000, 1 << 28, 4, 2, per_string_launches=True)
