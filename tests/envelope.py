"""Tolerance checks of the FP32-mixed parity tests: each prints the measured error beside its
bound (visible with pytest -s), so that the envelopes can be kept near the measurements."""


def check(label, err, bound):
    print("envelope %-48s measured %.3e  bound %.1e" % (label, err, bound))
    assert err <= bound, (label, err, bound)
