"""(Cin, Cout) of the twelve 3x3 layers of the learned initialiser, in parameter order
(encoder e0a e0b e1a e1b e2a e2b e3a e3b, decoder d2 d1 d0, head), as built by
libfb.so; each layer's parameters are weights [Cout][3][3][Cin] then biases [Cout]."""
LAYERS = [(8, 32), (32, 32), (32, 64), (64, 64), (64, 96), (96, 96), (96, 128), (128, 128),
          (224, 96), (160, 64), (96, 32), (32, 8)]
