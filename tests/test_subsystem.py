"""The sampled full-size parity test steps only the samples' n-hop
neighbourhoods with the oracle.  This pins that method on the CPU: after n
steps, the oracle on the n-hop sub-system gives the samples exactly the
whole-system result (a mass depends only on masses within n springs of it),
and one hop fewer is not enough."""
import importlib.util
import os

import numpy as np

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def fullsize_helpers():
    spec = importlib.util.spec_from_file_location("fullsize", os.path.join(HERE, "test_gpu_fullsize.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_n_hop_subsystem_is_exact_for_the_samples(ora):
    fs = fullsize_helpers()
    s = synth.throughput_lattice(n=16)
    p = fs.f32p(synth.throughput_params())
    N = s["x"].shape[0]
    samples = np.array([0, 15, 16 * 16 * 5 + 37, 2000, N - 1])
    xa, va = ora.run(s, p, 4)
    sub, remap = fs.subsystem(s, fs.hops(s["ij"], N, samples, 4))
    assert sub["x"].shape[0] < N
    xo, vo = ora.run(sub, p, 4)
    assert np.array_equal(xo[remap[samples]], xa[samples])
    assert np.array_equal(vo[remap[samples]], va[samples])
    # three hops are not enough for four steps: some free sample differs
    sub3, remap3 = fs.subsystem(s, fs.hops(s["ij"], N, samples, 3))
    x3, _ = ora.run(sub3, p, 4)
    assert not np.array_equal(x3[remap3[samples]], xa[samples])
