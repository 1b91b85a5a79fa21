"""td_segment_load rejects wrong, inconsistent and truncated checkpoint files
before any device work (so these run without a GPU)."""
import ctypes
import struct

import numpy as np
import pytest

HDR = "<8sIIqqqqdiiddQQ"          # the 96-byte header of the checkpoint format
MAGIC = b"TDSEGCK1"


def _lib():
    from paper_2603_06010_b300 import td
    return td


def _header(n=300, nk=300, nkp=512, flags=1, factored=1, op_blocks=None, logm=0, payload=None, version=1,
            magic=MAGIC):
    m = nkp // 256
    if op_blocks is None:
        op_blocks = 8 * m * (m + 1) // 2
    if payload is None:
        payload = n * 8 + nk * 4 + (op_blocks * 4 * 256 * 32 * 2 if flags & 1 else 0)
    return struct.pack(HDR, magic, version, flags, n, nk, nkp, op_blocks, -1.5, logm, factored, 0.0, 0.0,
                       payload, 0), payload


def _load(td, path):
    h = ctypes.c_void_p()
    st = td.lib().td_segment_load(str(path).encode(), None, ctypes.byref(h))
    return st, h.value, td.lib().td_last_error().decode()


def _write(path, header, payload_bytes, t=None, n=300):
    body = bytearray(payload_bytes)
    acf = np.zeros(n)
    acf[0] = 1.0
    body[:n * 8] = acf.tobytes()
    if t is not None:
        body[n * 8:n * 8 + 4 * len(t)] = np.asarray(t, np.int32).tobytes()
    path.write_bytes(header + bytes(body))


def test_header_is_96_bytes():
    assert struct.calcsize(HDR) == 96


@pytest.mark.parametrize("case,needle", [
    ("missing", "cannot open"),
    ("short", "shorter than a checkpoint header"),
    ("magic", "magic"),
    ("version", "version"),
    ("flags0", "flags"),
    ("flags8", "flags"),
    ("nk_gt_n", "inconsistent sizes"),
    ("nkp", "inconsistent sizes"),
    ("op_blocks", "operator size"),
    ("payload", "payload size"),
    ("truncated", "file size"),
    ("longer", "file size"),
    ("unordered", "kept indices"),
    ("gs_len", "GSCE length"),
    ("factored_no_op", "without its operator"),
])
def test_bad_checkpoint_rejected_before_device_work(tmp_path, case, needle):
    td = _lib()
    p = tmp_path / "seg.ckpt"
    t_ok = np.arange(300)
    if case == "missing":
        pass
    elif case == "short":
        p.write_bytes(b"TDSEG")
    else:
        kw = {"magic": {"magic": b"XXXXXXXX"}, "version": {"version": 2}, "flags0": {"flags": 0},
              "flags8": {"flags": 8}, "nk_gt_n": {"nk": 301}, "nkp": {"nkp": 256}, "op_blocks": {"op_blocks": 23},
              "gs_len": {"flags": 5, "logm": 9}, "factored_no_op": {"flags": 4, "factored": 1, "logm": 11},
              }.get(case, {})
        hdr, payload = _header(**kw)
        if case == "payload":
            hdr, _ = _header(payload=payload + 8)
        size = payload - 1 if case == "truncated" else (payload + 1 if case == "longer" else payload)
        t = t_ok.copy()
        if case == "unordered":
            t[10], t[11] = t[11], t[10]
        _write(p, hdr, size, t=t)
    st, h, msg = _load(td, p)
    assert st == td.TD_ERR_INVALID, (case, st, msg)
    assert h is None
    assert needle in msg, (case, msg)


def test_load_argument_errors():
    td = _lib()
    L = td.lib()
    h = ctypes.c_void_p()
    assert L.td_segment_load(None, None, ctypes.byref(h)) == td.TD_ERR_INVALID
    assert L.td_segment_load(b"", None, ctypes.byref(h)) == td.TD_ERR_INVALID
    assert L.td_segment_load(b"x", None, None) == td.TD_ERR_INVALID
    assert L.td_segment_save(None, b"x", None) == td.TD_ERR_INVALID
