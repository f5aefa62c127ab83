"""Host-side check of the GPU FFT schedules: every (L, E, radices) entry of passes.cuh is
run through a numpy model of the kernels' Stockham stage indexing (the gather, twiddle,
scatter and pruning rules of fft_core.cuh) and compared with numpy's FFT.  This checks
the index arithmetic that decides which HBM rows a pass reads and writes, before any
kernel runs on a GPU."""
import os
import re

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
PASSES = os.path.join(os.path.dirname(HERE), "paper_1612_01799_gb300", "csrc", "passes.cuh")


def schedules():
    with open(PASSES) as f:
        text = f.read()
    out = []
    for m in re.finditer(r"GSP_FFT_CFG\((\d+),\s*(\d+),\s*([\d,\s]+)\);", text):
        L, E = int(m.group(1)), int(m.group(2))
        rs = [int(x) for x in m.group(3).split(",")]
        out.append((L, E, rs))
    return out


def stockham(x, L, E, radices, direction, prune_in, prune_out):
    """Model of Stages::run for one column.  Returns the output rows written (dict)."""
    P = L // E
    data = {i: x[i] for i in range(L)}          # readable rows of the current input
    NS = 1
    written = {}
    for s, R in enumerate(radices):
        first, last = s == 0, s == len(radices) - 1
        assert E % R == 0 and L % (NS * R) == 0
        out = {}
        for q in range(P):
            for b in range(E // R):
                j = q + P * b
                v = []
                for r in range(R):
                    row = j + r * (L // R)
                    if first and prune_in and 2 * r >= R:
                        v.append(0.0)
                    else:
                        assert 0 <= row < L
                        v.append(data[row])
                v = np.array(v, dtype=complex)
                k = j % NS
                tw = np.exp(direction * 2j * np.pi * np.arange(R) * k / (NS * R))
                v = v * tw
                n = np.arange(R)
                v = np.exp(direction * 2j * np.pi * np.outer(n, n) / R) @ v
                base = (j // NS) * NS * R + (j % NS)
                for r in range(R):
                    row = base + r * NS
                    if last and prune_out and 2 * r >= R:
                        continue
                    assert row not in out, "row written twice"
                    out[row] = v[r]
        data = out
        NS *= R
    return data


@pytest.mark.parametrize("L,E,radices", schedules())
def test_schedule_is_a_dft(L, E, radices):
    assert int(np.prod(radices)) == L
    assert radices[0] % 2 == 0 and radices[-1] % 2 == 0
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    # full forward and inverse
    y = stockham(x, L, E, radices, -1, False, False)
    assert sorted(y) == list(range(L))
    assert np.allclose([y[i] for i in range(L)], np.fft.fft(x), atol=1e-10)
    y = stockham(x, L, E, radices, +1, False, False)
    assert np.allclose([y[i] for i in range(L)], np.fft.ifft(x) * L, atol=1e-10)
    # forward with the upper half of the input zero (never read)
    xp = x.copy()
    xp[L // 2:] = np.nan                      # a read of a pruned row would poison the result
    y = stockham(xp, L, E, radices, -1, True, False)
    ref = np.fft.fft(np.concatenate([x[:L // 2], np.zeros(L - L // 2)]))
    assert np.allclose([y[i] for i in range(L)], ref, atol=1e-10)
    # inverse keeping exactly the lower half of the outputs
    y = stockham(x, L, E, radices, +1, False, True)
    assert sorted(y) == list(range(L // 2))
    assert np.allclose([y[i] for i in range(L // 2)], (np.fft.ifft(x) * L)[:L // 2], atol=1e-10)


@pytest.mark.parametrize("L,E,radices", schedules())
def test_z_pass_chain(L, E, radices):
    """The fused z pass: forward with the schedule (upper input half zero), a pointwise
    symbol, then the inverse with the radices reversed keeping the lower output half.
    The inverse's first stage has the forward's last radix and reads exactly the rows the
    forward's last stage left in each thread, so no exchange is needed between them."""
    rng = np.random.default_rng(L + 1)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    x[L // 2:] = 0
    g = rng.standard_normal(L)
    y = stockham(x, L, E, radices, -1, True, False)
    P = L // E
    R_last = radices[-1]
    # rows held by thread q after the forward's last stage = rows its first inverse stage gathers
    for q in range(P):
        held = {q + P * b + r * (L // R_last) for b in range(E // R_last) for r in range(R_last)}
        assert len(held) == E
    z = stockham(np.array([y[i] * g[i] for i in range(L)]), L, E, radices[::-1], +1, False, True)
    ref = np.fft.ifft(np.fft.fft(x) * g) * L
    assert np.allclose([z[i] for i in range(L // 2)], ref[:L // 2], atol=1e-9)


def test_every_supported_n_has_both_schedules():
    lengths = {L for L, _, _ in schedules()}
    with open(PASSES) as f:
        m = re.search(r"#define GSP_SUPPORTED_N\(X\)\s*\\\s*(.*)", f.read())
    ns = [int(v) for v in re.findall(r"X\((\d+)\)", m.group(1))]
    for n in ns:
        assert n in lengths and 2 * n in lengths, n
