"""The learned cost model's arithmetic in fp64 -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and bench.py's CPU-baseline leg may import this.
It shares no code with the CUDA library.

The paper fixes q from log_sigma(rm) and k by a closed form (Section 3.2);
it has no learned model, so nothing here restates the paper.  What it
restates are textbook definitions, in plain numpy, slow and obvious:

  forward      a multilayer perceptron 8 -> 64 -> 64 -> 1 with ReLU hidden
               units and a linear output, on standardised inputs
               x~ = (x - mean) / std:
                   h1 = relu(W1 x~ + b1)
                   h2 = relu(W2 h1 + b2)
                   f  = w3 . h2 + b3
  loss         mean squared error against standardised targets
               y~ = (y - y_mean) / y_std:  L = (1/N) sum_s (f_s - y~_s)^2
  gradient     dL/dtheta by the chain rule, written out by hand (reverse
               order of forward; ReLU'(z) taken as 1 for z > 0, else 0)
  adam_step    Adam (Kingma and Ba, 2015): m = b1 m + (1 - b1) g,
               v = b2 v + (1 - b2) g^2, m^ = m / (1 - b1^t),
               v^ = v / (1 - b2^t), theta -= lr m^ / (sqrt(v^) + eps)

Parameter layout (one flat vector, the same order as the library's):
W1 (64 x 8, row j = hidden unit j), b1 (64), W2 (64 x 64, row j = unit j of
the second layer), b2 (64), w3 (64), b3 (1): 4801 numbers.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss
against the hand-written gradient; a network with one live path whose output
is computed by hand; a purely linear regime whose least-squares optimum is
known in closed form; and the first Adam step, which moves every parameter
by lr * g / (|g| + eps) exactly.
"""
import numpy as np

N_IN = 8
N_HID = 64
SIZES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("w3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    """Flat parameter vector -> dict of arrays (views)."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAMS,)
    out, at = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[at:at + n].reshape(shape)
        at += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1)
                           for name, _ in SIZES])


def standardise(X, mean, std):
    return (np.asarray(X, np.float64) - np.asarray(mean, np.float64)) / np.asarray(std, np.float64)


def forward(theta, Xs):
    """Outputs f (N,) and the hidden activations, for standardised inputs Xs (N, 8)."""
    p = unpack(theta)
    Xs = np.asarray(Xs, np.float64)
    z1 = Xs @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    f = h2 @ p["w3"] + p["b3"][0]
    return f, (z1, h1, z2, h2)


def loss(theta, Xs, ys):
    f, _ = forward(theta, Xs)
    d = f - np.asarray(ys, np.float64)
    return float(np.mean(d * d))


def gradient(theta, Xs, ys):
    """(loss, dL/dtheta) with the chain rule written out layer by layer."""
    p = unpack(theta)
    Xs = np.asarray(Xs, np.float64)
    ys = np.asarray(ys, np.float64)
    N = Xs.shape[0]
    f, (z1, h1, z2, h2) = forward(theta, Xs)
    d = f - ys
    L = float(np.mean(d * d))
    df = 2.0 * d / N                        # dL/df_s
    g = {}
    g["w3"] = df @ h2                       # sum_s df_s h2_s
    g["b3"] = np.array([df.sum()])
    dh2 = np.outer(df, p["w3"])             # dL/dh2
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1                    # sum_s dz2_s (outer) h1_s
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ Xs
    g["b1"] = dz1.sum(axis=0)
    return L, pack(g)


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; t is the step number after the update (1, 2, ...).
    Returns (theta, m, v)."""
    grad = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta = np.asarray(theta, np.float64) - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def regret(pred, measured):
    """Regret of choosing argmin(pred) among configurations whose measured
    times are `measured`: t(chosen) / min(t) - 1."""
    pred = np.asarray(pred)
    measured = np.asarray(measured, np.float64)
    return float(measured[int(np.argmin(pred))] / measured.min() - 1.0)
