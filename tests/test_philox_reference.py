"""Pin the oracle's Philox4x32-10 to an independent library implementation.

Philox4x32-10 is the published counter-based generator of Salmon et al.
(SC'11).  Triton ships its own implementation of the same generator
(triton.language.philox; key = the 64-bit seed split into low/high words,
counter = four 32-bit words, ten rounds).  Its CPU interpreter evaluates it
without a GPU, so the oracle's outputs can be compared word for word.  This is
a test-only use of the library as a reference for the published algorithm.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np

SCRIPT = textwrap.dedent(r'''
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(ctr, out, seed, n: tl.constexpr):
        i = tl.arange(0, n)
        c0 = tl.load(ctr + 4 * i + 0).to(tl.uint32, bitcast=True)
        c1 = tl.load(ctr + 4 * i + 1).to(tl.uint32, bitcast=True)
        c2 = tl.load(ctr + 4 * i + 2).to(tl.uint32, bitcast=True)
        c3 = tl.load(ctr + 4 * i + 3).to(tl.uint32, bitcast=True)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out + 4 * i + 0, a.to(tl.int32, bitcast=True))
        tl.store(out + 4 * i + 1, b.to(tl.int32, bitcast=True))
        tl.store(out + 4 * i + 2, c.to(tl.int32, bitcast=True))
        tl.store(out + 4 * i + 3, d.to(tl.int32, bitcast=True))

    seed = int(sys.argv[1])
    ctr = np.load(sys.argv[2])
    n = ctr.shape[0]
    out = torch.zeros(n * 4, dtype=torch.int32)
    k[(1,)](torch.from_numpy(ctr.view(np.int32).ravel().copy()), out, seed, n)
    np.save(sys.argv[3], out.numpy().view(np.uint32).reshape(n, 4))
''')


def test_oracle_philox_equals_triton_philox(orc, tmp_path):
    rng = np.random.default_rng(5)
    n = 256
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:8] = [[s, 0, p, 0xFFFFFFFF] for s in range(4) for p in (0, 2)]  # init / division style counters
    for seed in (0x0123_4567_89AB_CDEF, 42):
        cpath, opath, spath = tmp_path / "c.npy", tmp_path / "o.npy", tmp_path / "k.py"
        np.save(cpath, ctr)
        spath.write_text(SCRIPT)
        env = dict(os.environ, TRITON_INTERPRET="1")
        subprocess.check_call([sys.executable, str(spath), str(seed), str(cpath), str(opath)], env=env,
                              timeout=600)
        want = np.load(opath)
        got = orc.philox(ctr, seed)
        assert np.array_equal(got, want)
