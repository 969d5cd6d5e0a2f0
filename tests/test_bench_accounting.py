"""Host-side accounting of the benchmark: the algorithmic FLOP counts behind
the search kernel's roofline figure (bench.py: flops_per_sim, pow_products,
pulse_end_flops), checked against counts derived independently from the
structure of the propagators; the key of the DRAM traffic record; and the
summary of the clock samples taken during the timed region.

Within one input phase the plant's one-sample RK4 propagator has the block
structure of the state (theta, omega, x, y | F_a, F_n): the mechanical rows
depend on all six states, each activation only on itself.  The kernel keeps
both phases' propagators with one shared mechanical block (the phases differ
only in the activation time constants, hence in the coupling columns and the
activation diagonal).  Counts use FMA = 2 FLOP."""
import numpy as np

import bench

MECH, ACT = 4, 2


def structure():
    """Structural non-zeros of one phase's 6x6 increment matrix."""
    s = np.zeros((6, 6), bool)
    s[:MECH, :] = True                     # mechanical rows: every state
    s[MECH, MECH] = s[MECH + 1, MECH + 1] = True   # activations: first order, decoupled
    return s


def product_flops(sa, sb, entries):
    """FLOPs of R = A + B + A B on the given output entries (increment form of
    (I + A)(I + B) - I), counting one add per output entry for A + B where
    either is non-zero and one FMA per structural term of A B."""
    fl = 0
    for (i, j) in entries:
        if sa[i, j] or sb[i, j]:
            fl += 1 if (sa[i, j] and sb[i, j]) else 0   # a + b (a lone term needs no add)
        fl += 2 * int(np.sum(sa[i, :] & sb[:, j]))
    return fl


def test_one_sample_update_is_26_fma_plus_the_residual():
    s = structure()
    assert int(s.sum()) == 26
    # per integrated sample: the block update, then (theta - y)^2 accumulated:
    # a subtraction and one FMA
    assert 2 * int(s.sum()) + 3 == 55
    assert bench.flops_per_sim(101, 0, 10) - bench.flops_per_sim(100, 0, 10) == 55


def test_propagator_product_count():
    """Both phases' increment matrices multiplied at once: the mechanical
    block (rows and columns 0-3) once, the coupling columns and the
    activation diagonal per phase."""
    s = structure()
    mech = [(i, j) for i in range(MECH) for j in range(MECH)]
    per_phase = [(i, j) for i in range(MECH) for j in range(MECH, 6)] + [(MECH, MECH), (MECH + 1, MECH + 1)]
    total = product_flops(s, s, mech) + 2 * product_flops(s, s, per_phase)
    assert total == 332


def _powering(n):
    """Left-to-right binary powering of x = q: square, then multiply by q
    when the next bit is set.  Returns (products, exponent reached)."""
    e, products = 1, 0
    for b in range(n.bit_length() - 2, -1, -1):
        e, products = 2 * e, products + 1
        if (n >> b) & 1:
            e, products = e + 1, products + 1
    return products, e


def test_powering_products_match_the_binary_method():
    for n in range(1, 1025):
        products, e = _powering(n)
        assert e == n
        assert bench.pow_products(n) == products
    # the sample rates of the workloads: 10, 20 and 40 substeps per sample
    assert [bench.pow_products(bench.nsub_for(fs)) for fs in (1000.0, 500.0, 250.0)] == [4, 5, 6]


def plant_structure():
    """Structural non-zeros of the plant matrix A in deviation coordinates
    (around the phase's equilibrium, so the neural input drops out):
    theta' = omega (a unit coefficient), omega' from theta, omega, x, y
    (series tensions, globe viscosity and elasticity), x' from theta, x, F_a,
    y' from theta, y, F_n, and F' = -F / tau for each activation."""
    rows = {0: [1], 1: [0, 1, 2, 3], 2: [0, 2, 4], 3: [0, 3, 5], 4: [4], 5: [5]}
    return rows


def apply_flops(rows):
    """FLOPs of v -> A v: a row of k coefficients is one product and k - 1
    FMAs (2k - 1), except theta' = omega, which is a copy."""
    return sum(0 if r == 0 else 2 * len(c) - 1 for r, c in rows.items())


def test_pulse_end_interval_count():
    """The sample that holds the pulse end: nsub - 1 single-substep block
    updates, two RK4 steps around the switch, the split step lengths and the
    equilibrium shift, less the one-sample update already counted for that
    sample.  For a linear system one RK4 step is e + hA(e + hA/2(e + hA/3(e +
    hA/4 e))): four applications of A, each followed by six FMAs, and the three
    level coefficients h/2, h/3, h/4."""
    a = apply_flops(plant_structure())
    assert a == 19
    rk4_step = 4 * (a + 6 * 2) + 3
    assert rk4_step == 127
    update = 2 * int(structure().sum())
    for nsub in (1, 10, 20, 40, 640):
        assert bench.pulse_end_flops(nsub) == update * (nsub - 1) + 2 * rk4_step + 2 + 6 - update
    # the stage-by-stage comparison figure: four derivative evaluations with
    # the neural input (one more FMA per activation row: 21), three stage
    # states and the final combination (168 per substep)
    assert 4 * (a + 2) + 3 * 6 * 2 + 6 * 4 * 2 == 168
    assert bench.rk4_stage_flops_per_sim(11, 10) == 168 * 10 * 10


def test_traffic_record_key_ignores_comments_only():
    """The DRAM traffic record is keyed by a digest of the kernel sources
    that a comment edit leaves alone and a code edit changes."""
    src = ["int f(int a) {  // add one\n  return a + 1;\n}\n", "// header\n#pragma once\n"]
    same = ["int f(int a) {  // add one to a\n\n  return a + 1;   \n}\n", "// header, reworded\n#pragma once\n"]
    code = ["int f(int a) {  // add one\n  return a + 2;\n}\n", "// header\n#pragma once\n"]
    assert bench.source_code_digest(src) == bench.source_code_digest(same)
    assert bench.source_code_digest(src) != bench.source_code_digest(code)
    assert len(bench.kernel_hash()) == 64


def test_clock_samples_summary():
    """nvidia-smi samples during the timed region: the median SM clock and
    every throttle reason seen active; malformed lines are skipped."""
    lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1400.1, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    d = bench.parse_clock_samples(lines)
    assert d == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}
    assert bench.parse_clock_samples([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_surrogate_training_flops_count_the_products_formed():
    # forward: four 512 x 512 layers and the 18-wide output layer; backward:
    # the output layer's weight gradient and dH3, four hidden weight
    # gradients, error products for layers 3, 2, 1 only
    fwd = 4 * 512 * 512 + 18 * 512
    bwd = 2 * 18 * 512 + 4 * 512 * 512 + 3 * 512 * 512
    assert bench.MLP_TRAIN_FLOP_PER_SAMPLE == 2 * (fwd + bwd)
    assert bench.MLP_TRAIN_FLOP_PER_SAMPLE < 3 * 2 * fwd
