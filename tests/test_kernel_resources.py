"""Register budget of the interior kernels (host-side compilation, no GPU).

The interior kernel is bound by HBM bandwidth only while enough warps are in
flight; its default launch shapes are sized so that their registers fit
(variant 0: 6 blocks of 128 threads per SM, at most 80 registers; FP64
storage's variant 2: 4 blocks, 128 registers; BFP13 storage's variant 4: 6
blocks with u one row ahead; the batched kernel's variant 5: 5 blocks, 96
registers; the frame kernel of two steps per sweep: 6 blocks; the two-step
kernel: 5 blocks, 96 registers).  A spill to local memory inside the row loop
costs far more than the bytes it saves (a 20-byte spill once took the BF16
kernel from 1.38 to 2.02 ms per 8192^2 launch), so every default shape must
compile without one.  ptxas prints, per kernel, the registers it used and
the bytes it spilled (-Xptxas -v)."""
import re
import subprocess

import pytest

from paper_2301_00228_gb300 import build as B

# (kernel name prefix, policy in the mangled name, (MINB, UVD) of the default variant)
DEFAULTS = [
    ("bulk_kernel", "PopDirectIfE", (6, 2)),
    ("bulk_kernel", "PopNeq16I6__halfE", (6, 2)),
    ("bulk_kernel", "PopNeq16I13__nv_bfloat16E", (6, 2)),
    ("bulk_kernel", "PopBfp13", (6, 1)),
    ("bulk_kernel", "PopDirectIdE", (4, 2)),
    ("bulk_batch_kernel", "PopDirectIfE", (5, 1)),
    ("bulk_batch_kernel", "PopNeq16I6__halfE", (5, 1)),
    ("bulk_batch_kernel", "PopNeq16I13__nv_bfloat16E", (5, 1)),
    ("bulk_batch_kernel", "PopBfp13", (5, 1)),
    ("frame_kernel", "PopBfp13", (6, 1)),
    ("frame_kernel", "PopDirectIfE", (6, 2)),
    ("pair_kernel", "PopDirectIfE", (5, None)),
    ("pair_kernel", "PopNeq16I6__halfE", (5, None)),
    ("pair_kernel", "PopBfp13", (5, None)),
]


@pytest.fixture(scope="module")
def ptxas_report(tmp_path_factory):
    try:
        nvcc = B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("ptxas") / "lbps_kernels.o"
    cmd = [nvcc] + B.ARCH + ["-O3", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-I", str(B.INCLUDE),
                             "-I", str(B.CSRC), "-Xptxas", "-v", "-c", str(B.CSRC / "lbps_kernels.cu"), "-o", str(out)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    # kernel -> (registers, spill store bytes, spill load bytes)
    info, cur = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"(?:Compiling entry function|Function properties for) '?(_Z\w+)", line)
        if m:
            cur = m.group(1)
            info.setdefault(cur, [None, None, None])
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and cur:
            info[cur][1:] = [int(m.group(1)), int(m.group(2))]
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            info[cur][0] = int(m.group(1))
    return info


@pytest.mark.parametrize("kernel,policy,shape", DEFAULTS)
def test_default_shapes_do_not_spill(ptxas_report, kernel, policy, shape):
    minb, uvd = shape
    tail = f"ELi{minb}EE" if uvd is None else f"ELi{minb}ELi{uvd}E"
    pat = re.compile(rf"\d{kernel}INS_\d+{policy}{tail}")
    hits = [(k, v) for k, v in ptxas_report.items() if pat.search(k)]
    assert len(hits) == 1, (kernel, policy, shape, len(hits))
    name, (regs, st, ld) = hits[0]
    assert regs is not None and regs <= 65536 // (128 * minb), (name, regs)
    assert (st, ld) == (0, 0), (name, st, ld)
