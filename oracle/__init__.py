"""FP64 CPU oracle for the structural-plasticity hot path — TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy implementations of what the paper's method
computes (Knight, Senk & Nowotny, "A flexible framework for structural plasticity in
GPU-accelerated sparse spiking neural networks"):

* `philox`     counter-based random numbers (Philox4x64-10, Salmon et al., SC'11),
* `classifier` LIF/ALIF recurrent classifier, leaky readout, e-prop eligibility traces
               and gradients in their forward (trace) form, L1 on the sign bitfield,
               Adam (Sec. 2.2.1, Eqs. for v, a, z, y, epsilon, e, Delta W),
* `deepr`      DEEP R bitfield initialisation, elimination, dormant redistribution and
               formation (Sec. 2.1.2, Fig. 2),
* `topo`       topographic map: correlated Poisson input, conductance LIF with
               exponential Euler, all-to-all STDP, parallel rewiring with the
               distance-dependent formation and weight-dependent elimination rules
               (Sec. 2.1.3, Fig. 3, Tab. 1-2).

Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / reference arm of
`bench.py` may import this package.  It shares no code with the CUDA library and never
imports it; the only module both sides use is `synth` (seeded inputs, none of the
method's arithmetic).

Parity status: every function here is pinned by a `-m "not gpu"` test against a
closed form, a library routine (numpy's Philox, torch autograd BPTT, torch.optim.Adam),
brute force on tiny inputs, invariants or statistical bounds, except the items listed
under "parity unpinned" in the individual module headers.
"""
