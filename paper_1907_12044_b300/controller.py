"""Initial weights of the learned Krylov controller (the network itself runs in libtdvp).

Layout (4866 float32): W1[8][64], b1[64], W2[64][64], b2[64], W3[64], b3 (Krylov-dimension head),
W4[64], b4 (acceptance head).  He-normal weights, zero biases, output bias 4 (a typical Krylov
dimension), acceptance weights zero (probability 1/2 before training), from a seed.
"""
import numpy as np

NIN, NH = 8, 64


def init_weights(seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, np.sqrt(2.0 / NIN), (NIN, NH)).ravel(), np.zeros(NH),
             rng.normal(0.0, np.sqrt(2.0 / NH), (NH, NH)).ravel(), np.zeros(NH),
             rng.normal(0.0, np.sqrt(1.0 / NH), NH), np.array([4.0]), np.zeros(NH), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)
