"""Small integer-only cases shared by the oracle regression fixture and the
GPU parity tests (inputs only; no expected values)."""
import synth

REGRESSION_CASES = ["u8x3-48x40-L3-T12000-r1", "u8x2-33x29-L4-T60-r2",
                    "u16x2-40x36-L5-T4096-r3", "u8x1-31x17-L2-T10-r0",
                    "u8x4-20x24-L3-T20000-r1"]


def make_case(name):
    if name == "u8x3-48x40-L3-T12000-r1":
        return dict(tgt=synth.smooth_integer_guide(1, 40, 48, 3, step=4),
                    src=synth.smooth_integer_guide(2, 36, 44, 3, step=4),
                    style=synth.random_style(3, 36, 44), key_bits=4, levels=3,
                    threshold=12000, radius=1, seed=11)
    if name == "u8x2-33x29-L4-T60-r2":
        return dict(tgt=synth.smooth_integer_guide(4, 29, 33, 2, step=3),
                    src=synth.smooth_integer_guide(5, 30, 30, 2, step=3),
                    style=synth.random_style(6, 30, 30), key_bits=6, levels=4,
                    threshold=60, radius=2, seed=0xC0FFEE)
    if name == "u16x2-40x36-L5-T4096-r3":
        src = synth.identity_uv_guide(32, 48)
        tgt = synth.random_guide(7, 36, 40, 2, bits=16, low=0, high=47 * 32)
        return dict(tgt=tgt, src=src, style=synth.random_style(8, 32, 48), key_bits=8,
                    levels=5, threshold=4096, radius=3, seed=5)
    if name == "u8x1-31x17-L2-T10-r0":
        return dict(tgt=synth.random_guide(9, 17, 31, 1), src=synth.random_guide(10, 13, 11, 1),
                    style=synth.random_style(11, 13, 11), key_bits=8, levels=2,
                    threshold=10, radius=0, seed=1)
    if name == "u8x4-20x24-L3-T20000-r1":
        return dict(tgt=synth.smooth_integer_guide(12, 24, 20, 4, step=2),
                    src=synth.smooth_integer_guide(13, 16, 18, 4, step=2),
                    style=synth.random_style(14, 16, 18), key_bits=3, levels=3,
                    threshold=20000, radius=1, seed=99)
    raise KeyError(name)
