"""Reference definition of the surrogate's input features (FP64).

TEST INFRASTRUCTURE ONLY (imported by the tests, never by the product).

The surrogate maps a recorded saccade to an OPC estimate; the paper has no
learned part, so the features are this library's own definition:

* work in the positive frame: a saccade whose end fixation lies below its
  start fixation is mirrored (every position negated), so every feature
  vector describes a movement from a0 = sign * theta_start up to
  af = sign * theta_end;
* resample 257 points 1 ms apart from the onset sample: point i sits at the
  fractional sample index s_i = onset + i * fs / 1000, held at the last
  sample L - 1 once the window ends, and takes the linear interpolation of the
  two samples around it;
* position feature i (i < 256) = (sign * y(s_i) - a0) / A with the amplitude
  A = max(af - a0, 0.5 deg), so the start fixation maps to 0 and the end
  fixation to 1;
* velocity feature i (i < 256) = 10 * (position i+1 - position i), the
  per-millisecond difference scaled to order one, except the last, which is 0.

Output: 512 features, positions 0..255 then velocities 256..511.  Pinned in
the tests on ramps, constants and mirrored traces, whose features are known in
closed form.
"""
from __future__ import annotations

import math

import numpy as np

POINTS = 256


def featurize(y, fs, onset, theta_start, theta_end) -> np.ndarray:
    y = np.asarray(y, dtype=np.float64)
    L = len(y)
    sign = -1.0 if theta_end < theta_start else 1.0
    a0, af = sign * float(theta_start), sign * float(theta_end)
    amp = max(af - a0, 0.5)
    pos = np.zeros(POINTS + 1)
    for i in range(POINTS + 1):
        s = min(onset + i * float(fs) / 1000.0, L - 1)
        k0 = int(math.floor(s))
        k1 = min(k0 + 1, L - 1)
        w = s - k0
        pos[i] = (sign * ((1.0 - w) * y[k0] + w * y[k1]) - a0) / amp
    vel = 10.0 * (pos[1:] - pos[:-1])
    vel[POINTS - 1] = 0.0
    return np.concatenate([pos[:POINTS], vel])
